// mrq_sci.cu - heat-bath selected-CI reference phi0 built on the device (Sec. II D: a selected-CI
// reference in the spirit of heat-bath CI), followed by the semicanonical rotation of the core and
// virtual orbitals that Dyall's H_D assumes (Sec. II C), behind mrq_sci_reference (include/mrq.h).
//
// The reference lives in the product space S x S of selected alpha and beta occupation strings of
// the active space (Sz = 0), with the core-averaged active Hamiltonian
//     H = E_core + sum_tu h_tu E_tu + 1/2 sum_tuvw (tu|vw) (E_tu E_vw - delta_uv E_tw),
//     h = h1 + sum_i [2(..|ii) - (.i|i.)] over the doubly occupied core.
// Selection: solve in the product space of the n_seed strings of lowest same-spin energy, score
// every string s' by max_s |H^ss_s's| sqrt(w_s) (w_s: the weight of string s in that solution, H^ss
// the one-spin part of H), keep the n_strings best and solve again in their product space.
//
// Device layout (all FP64 unless stated):
//   strings      nstr uint32 occupation masks, lexicographic order of the combinations
//   g            (tu|vw) of the active space, na^4, index ((t na + u) na + v) na + w
//   Hss rows     CSR over the selected strings: (column, element) of every selected string within a
//                double replacement (the one-spin part, diagonal included)
//   os lists     per selected string J, the (I, t, u, sign) with E_tu |I> = sign |J>, I selected,
//                t = u included; k-major (entry k of every J contiguous) so a warp's reads coalesce
//   vectors      C[Ia][Ib] row-major, m^2 long; Davidson keeps max_sub of them and their images
// The sigma vector is one kernel (block per alpha string Ja, threads over Jb):
//   s[Ja,Jb] = E_core C + sum_Ia Hss[Ja,Ia] C[Ia,Jb] + sum_Ib Hss[Jb,Ib] C[Ja,Ib]
//            + sum_{(Ia,tu,sa) in L(Ja)} sum_{(Ib,vw,sb) in L(Jb)} sa sb (tu|vw) C[Ia,Ib].
// The Davidson driver runs on the host over device BLAS-1 kernels; only the subspace matrix (at
// most max_sub^2 numbers) and its eigenproblem live on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/mrq.h"
#include "mrq_internal.h"

namespace {

#define SCK(call)                                                                                        \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            return mrq_internal_fail(ctx, e_ == cudaErrorMemoryAllocation ? MRQ_OOM : MRQ_CUDA_ERROR,    \
                                     "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

constexpr int SCI_MAX_STR = 4096;               // selected strings per spin
constexpr long long SCI_MAX_SPACE = 1 << 16;    // strings of the full one-spin space (ranked in O(nstr^2))
constexpr int SCI_MAX_SUB = 64;

// ---------------------------------------------------------------------------- integrals

__host__ __device__ inline long long pidx(long long p, long long q) { return p >= q ? p * (p + 1) / 2 + q : q * (q + 1) / 2 + p; }
__host__ __device__ inline long long eidx(int p, int q, int r, int s) {
    const long long a = pidx(p, q), b = pidx(r, s);
    return pidx(a, b);
}

// active integrals g[t][u][v][w] = (tu|vw), core-averaged one-electron h[t][u] and the constant
// E_core = e_nuc + sum_i 2 h_ii + sum_ij [2(ii|jj) - (ij|ji)]
__global__ void k_sci_active(const double* __restrict__ h1, const double* __restrict__ eri, int n, int nc, int na,
                             double e_nuc, double* __restrict__ g, double* __restrict__ h, double* __restrict__ ecore) {
    const long long na2 = (long long)na * na, na4 = na2 * na2;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < na4 + na2 + 1;
         x += (long long)gridDim.x * blockDim.x) {
        if (x < na4) {
            const int w = (int)(x % na), v = (int)((x / na) % na), u = (int)((x / na2) % na), t = (int)(x / (na2 * na));
            g[x] = eri[eidx(nc + t, nc + u, nc + v, nc + w)];
        } else if (x < na4 + na2) {
            const int tu = (int)(x - na4), t = tu / na, u = tu % na, p = nc + t, q = nc + u;
            double v = h1[p * n + q];
            for (int i = 0; i < nc; i++) v += 2.0 * eri[eidx(p, q, i, i)] - eri[eidx(p, i, i, q)];
            h[tu] = v;
        } else {
            double e = e_nuc;
            for (int i = 0; i < nc; i++) {
                e += 2.0 * h1[i * n + i];
                for (int j = 0; j < nc; j++) e += 2.0 * eri[eidx(i, i, j, j)] - eri[eidx(i, j, j, i)];
            }
            *ecore = e;
        }
    }
}

// ---------------------------------------------------------------------------- strings

struct Binom {
    unsigned long long c[33][33];
};

// r-th combination of ne of na orbitals in lexicographic order of the sorted index tuples
__global__ void k_sci_unrank(Binom B, int na, int ne, long long nstr, unsigned* __restrict__ strs) {
    const long long r0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r0 >= nstr) return;
    unsigned long long r = (unsigned long long)r0;
    unsigned s = 0u;
    int x = 0;
    for (int j = 0; j < ne; j++) {
        for (;;) {
            const unsigned long long c = B.c[na - 1 - x][ne - 1 - j];
            if (r < c) break;
            r -= c;
            x++;
        }
        s |= 1u << x;
        x++;
    }
    strs[r0] = s;
}

__device__ __forceinline__ long long str_rank(const Binom& B, unsigned s, int na, int ne) {
    long long r = 0;
    int x = 0, j = 0;
    while (s) {
        const int b = __ffs(s) - 1;
        s &= s - 1;
        for (int y = x; y < b; y++) r += (long long)B.c[na - 1 - y][ne - 1 - j];
        x = b + 1;
        j++;
    }
    return r;
}

// (-1)^(occupied orbitals of s strictly between p and q)
__device__ __forceinline__ double between_sign(unsigned s, int p, int q) {
    const int lo = min(p, q), hi = max(p, q);
    const unsigned m = hi - lo > 1 ? ((1u << hi) - 1u) & ~((2u << lo) - 1u) : 0u;
    return (__popc(s & m) & 1) ? -1.0 : 1.0;
}

struct SciTabs {
    const double* g;     // na^4
    const double* h;     // na^2
    int na;
};

// one-spin diagonal: sum_i h_ii + 1/2 sum_{i,j in I} [(ii|jj) - (ij|ji)]
__device__ double ss_diag(const SciTabs& T, unsigned I) {
    const int na = T.na;
    double v = 0.0;
    for (unsigned a = I; a; a &= a - 1) {
        const int i = __ffs(a) - 1;
        v += T.h[i * na + i];
        for (unsigned b = I; b; b &= b - 1) {
            const int j = __ffs(b) - 1;
            v += 0.5 * (T.g[((i * na + i) * na + j) * na + j] - T.g[((i * na + j) * na + j) * na + i]);
        }
    }
    return v;
}

// <J| one-spin part |I> for I != J (Slater-Condon within one spin string)
__device__ double ss_offdiag(const SciTabs& T, unsigned I, unsigned J) {
    const unsigned x = I ^ J;
    const int d = __popc(x), na = T.na;
    if (d == 2) {
        const int i = __ffs(I & x) - 1, a = __ffs(J & x) - 1;
        double v = T.h[a * na + i];
        for (unsigned b = I; b; b &= b - 1) {
            const int j = __ffs(b) - 1;
            v += T.g[((a * na + i) * na + j) * na + j] - T.g[((a * na + j) * na + j) * na + i];
        }
        return between_sign(I, a, i) * v;
    }
    if (d == 4) {
        const unsigned rem = I & x, add = J & x;
        const int i = __ffs(rem) - 1, j = 31 - __clz(rem), a = __ffs(add) - 1, b = 31 - __clz(add);
        // <J|E_ai E_bj|I>: E_bj first (j -> b), then E_ai (i -> a)
        const unsigned K = (I & ~(1u << j)) | (1u << b);
        const double s = between_sign(I, b, j) * between_sign(K, a, i);
        return s * (T.g[((a * na + i) * na + b) * na + j] - T.g[((a * na + j) * na + b) * na + i]);
    }
    return 0.0;
}

__global__ void k_sci_diag(SciTabs T, const unsigned* __restrict__ strs, long long nstr, double* __restrict__ hd) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nstr) hd[r] = ss_diag(T, strs[r]);
}

// selection by rank: sel[i] = 1 when fewer than k entries precede i in the order (key descending
// when desc, else ascending; ties by index), i.e. the first k of a stable sort
__global__ void k_sci_rank_select(const double* __restrict__ key, long long n, long long k, int desc,
                                  unsigned char* __restrict__ sel) {
    extern __shared__ double tile[];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const double ki = i < n ? key[i] : 0.0;
    long long before = 0;
    for (long long base = 0; base < n; base += blockDim.x) {
        const long long j = base + threadIdx.x;
        tile[threadIdx.x] = j < n ? key[j] : 0.0;
        __syncthreads();
        const int cnt = (int)min((long long)blockDim.x, n - base);
        if (i < n) {
            for (int q = 0; q < cnt; q++) {
                const double kj = tile[q];
                const long long jj = base + q;
                const bool first = desc ? (kj > ki || (kj == ki && jj < i)) : (kj < ki || (kj == ki && jj < i));
                before += first ? 1 : 0;
            }
        }
        __syncthreads();
    }
    if (i < n) sel[i] = before < k ? 1 : 0;
}

// ordered compaction of the flagged indices (one block): out[c] = c-th flagged index for c < cap,
// *count = number flagged
__global__ void k_sci_compact(const unsigned char* __restrict__ flag, long long n, int* __restrict__ out, int cap,
                              int* __restrict__ count) {
    __shared__ long long part[1024];
    const long long per = (n + blockDim.x - 1) / blockDim.x;
    const long long lo = min(n, per * threadIdx.x), hi = min(n, lo + per);
    long long c = 0;
    for (long long i = lo; i < hi; i++) c += flag[i];
    part[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = 0;
        for (unsigned t = 0; t < blockDim.x; t++) {
            const long long v = part[t];
            part[t] = run;
            run += v;
        }
        *count = (int)run;
    }
    __syncthreads();
    long long pos = part[threadIdx.x];
    for (long long i = lo; i < hi; i++)
        if (flag[i]) {
            if (pos < cap) out[pos] = (int)i;
            pos++;
        }
}

// ---------------------------------------------------------------------------- product space

struct ProdDev {
    int m, na, cap;             // selected strings, active orbitals, os-list capacity per string
    const unsigned* str;        // m selected strings
    const int* row;             // m + 1 CSR offsets of the one-spin rows
    const int* col;
    const double* val;
    const unsigned* ent;        // os lists, k-major: ent[k m + J] = I | tu << 16 | sign << 31
    const int* cnt;             // m entries per list
    const double* g;            // na^4
    double ecore;
};

__device__ __forceinline__ unsigned os_pack(int I, int tu, double s) {
    return (unsigned)I | ((unsigned)tu << 16) | (s < 0.0 ? 0x80000000u : 0u);
}

// map[full index] = position in the selection (or -1), selected strings
__global__ void k_sci_select_map(const int* __restrict__ sel, int m, const unsigned* __restrict__ strs,
                                 int* __restrict__ map, unsigned* __restrict__ sstr) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < m) {
        map[sel[k]] = k;
        sstr[k] = strs[sel[k]];
    }
}

// one-spin rows: warp per selected string; pass 0 counts, pass 1 fills (columns in ascending order)
__global__ void k_sci_rows(const unsigned* __restrict__ sstr, const int* __restrict__ sel, int m, SciTabs T,
                           const double* __restrict__ hd, int pass, int* __restrict__ row, int* __restrict__ col,
                           double* __restrict__ val) {
    const int k = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (k >= m) return;
    const unsigned J = sstr[k];
    int pos = pass ? row[k] : 0;
    for (int base = 0; base < m; base += 32) {
        const int q = base + lane;
        const bool ok = q < m && __popc(J ^ sstr[q]) <= 4;
        const unsigned b = __ballot_sync(0xffffffffu, ok);
        if (pass && ok) {
            const int at = pos + __popc(b & ((1u << lane) - 1u));
            col[at] = q;
            val[at] = q == k ? hd[sel[k]] : ss_offdiag(T, sstr[q], J);
        }
        pos += __popc(b);
    }
    if (!pass && lane == 0) row[k] = pos;
}

// opposite-spin lists: thread per selected string J
__global__ void k_sci_oslists(const unsigned* __restrict__ sstr, int m, int na, int ne, Binom B,
                              const int* __restrict__ map, unsigned* __restrict__ ent, int* __restrict__ cnt) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    const unsigned J = sstr[k];
    int c = 0;
    for (unsigned a = J; a; a &= a - 1) {
        const int t = __ffs(a) - 1;
        for (int u = 0; u < na; u++) {
            if (u != t && ((J >> u) & 1u)) continue;
            const unsigned I = (J & ~(1u << t)) | (1u << u);
            const int idx = map[str_rank(B, I, na, ne)];
            if (idx < 0) continue;
            ent[(long long)c * m + k] = os_pack(idx, t * na + u, between_sign(I, t, u));   // E_tu: u -> t
            c++;
        }
    }
    cnt[k] = c;
}

// Davidson preconditioner: the diagonal of H in the product space
__global__ void k_sci_pdiag(ProdDev P, const int* __restrict__ sel, const double* __restrict__ hd,
                            double* __restrict__ diag) {
    const long long m = P.m, i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m * m) return;
    const int a = (int)(i / m), b = (int)(i % m), na = P.na;
    double v = P.ecore + hd[sel[a]] + hd[sel[b]];
    for (unsigned x = P.str[a]; x; x &= x - 1) {
        const int t = __ffs(x) - 1;
        for (unsigned y = P.str[b]; y; y &= y - 1) {
            const int u = __ffs(y) - 1;
            v += P.g[((t * na + t) * na + u) * na + u];
        }
    }
    diag[i] = v;
}

// sigma = H C in the product space (block per alpha string Ja, threads over beta strings Jb)
__global__ void __launch_bounds__(256) k_sci_sigma(ProdDev P, const double* __restrict__ C, double* __restrict__ out) {
    extern __shared__ unsigned la[];
    const int Ja = blockIdx.x, m = P.m, na2 = P.na * P.na;
    const int nla = P.cnt[Ja];
    for (int c = threadIdx.x; c < nla; c += blockDim.x) la[c] = P.ent[(long long)c * m + Ja];
    __syncthreads();
    const int r0 = P.row[Ja], r1 = P.row[Ja + 1];
    const double* Crow = C + (long long)Ja * m;
    for (int Jb = threadIdx.x; Jb < m; Jb += blockDim.x) {
        double acc = P.ecore * Crow[Jb];
        for (int q = r0; q < r1; q++) acc += P.val[q] * C[(long long)P.col[q] * m + Jb];
        for (int q = P.row[Jb], q1 = P.row[Jb + 1]; q < q1; q++) acc += P.val[q] * Crow[P.col[q]];
        const int nlb = P.cnt[Jb];
        for (int kb = 0; kb < nlb; kb++) {
            const unsigned eb = P.ent[(long long)kb * m + Jb];
            const double* grow = P.g + (long long)((eb >> 16) & 0x3ffu) * na2;     // (vw|tu) = (tu|vw)
            const double* Ccol = C + (eb & 0xffffu);
            double s = 0.0;
            for (int ka = 0; ka < nla; ka++) {
                const unsigned ea = la[ka];
                const double t = grow[(ea >> 16) & 0x3ffu] * Ccol[(long long)(ea & 0xffffu) * m];
                s += (ea >> 31) ? -t : t;
            }
            acc += (eb >> 31) ? -s : s;
        }
        out[(long long)Ja * m + Jb] = acc;
    }
}

// ---------------------------------------------------------------------------- BLAS-1 for Davidson

constexpr int DOT_BLOCKS = 304;

// part[r][b] = sum over block b's slice of A[r][i] y[i] (grid: DOT_BLOCKS x nrows)
__global__ void k_sci_dots(const double* __restrict__ A, long long N, const double* __restrict__ y,
                           double* __restrict__ part) {
    __shared__ double red[32];
    const int r = blockIdx.y;
    const double* a = A + (long long)r * N;
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        s += a[i] * y[i];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        part[(long long)r * gridDim.x + blockIdx.x] = t;
    }
}

__global__ void k_sci_dots_fin(const double* __restrict__ part, int nb, int nrows, double* __restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    double t = 0.0;
    for (int b = 0; b < nb; b++) t += part[(long long)r * nb + b];
    out[r] = t;
}

struct Coefs {
    double c[SCI_MAX_SUB];
};

// out = beta out + sum_j c_j A[j]
__global__ void k_sci_combine(const double* __restrict__ A, long long N, int k, Coefs cf, double beta,
                              double* __restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        double v = beta == 0.0 ? 0.0 : beta * out[i];
        for (int j = 0; j < k; j++) v += cf.c[j] * A[(long long)j * N + i];
        out[i] = v;
    }
}

// r = ax - e x; t = -r / (diag - e) with |diag - e| floored at 1e-8
__global__ void k_sci_precond(const double* __restrict__ x, const double* __restrict__ ax, const double* __restrict__ diag,
                              double e, long long N, double* __restrict__ r, double* __restrict__ t) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const double ri = ax[i] - e * x[i];
        double den = diag[i] - e;
        if (fabs(den) < 1e-8) den = 1e-8;
        r[i] = ri;
        t[i] = -ri / den;
    }
}

__global__ void k_sci_scale(double* __restrict__ x, long long N, double s) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        x[i] *= s;
}

// start vector: unit entry at the first minimum of the diagonal (found on the host) plus noise of
// amplitude 1e-4 from a counter hash, on top of an optional embedded guess
__global__ void k_sci_noise(double* __restrict__ x, long long N, unsigned long long salt) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull + salt;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        x[i] += 1e-4 * ((double)(z >> 11) * 0x1.0p-53 * 2.0 - 1.0);
    }
}

// index of the first entry of largest (mode 1: |x|) or smallest (mode 0: x) value, one block
__global__ void k_sci_argext(const double* __restrict__ x, long long N, int mode, long long* __restrict__ out) {
    __shared__ double bv[1024];
    __shared__ long long bi[1024];
    double v = 0.0;
    long long idx = -1;
    for (long long i = threadIdx.x; i < N; i += blockDim.x) {
        const double a = mode ? fabs(x[i]) : x[i];
        if (idx < 0 || (mode ? a > v : a < v)) {
            v = a;
            idx = i;
        }
    }
    bv[threadIdx.x] = v;
    bi[threadIdx.x] = idx;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if ((int)threadIdx.x < o) {
            const double a = bv[threadIdx.x + o];
            const long long j = bi[threadIdx.x + o];
            const double b = bv[threadIdx.x];
            const long long i = bi[threadIdx.x];
            const bool take = j >= 0 && (i < 0 || (mode ? a > b : a < b) || (a == b && j < i));
            if (take) {
                bv[threadIdx.x] = a;
                bi[threadIdx.x] = j;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = bi[0];
}

// ---------------------------------------------------------------------------- heat-bath selection

// w_s = (sum_b C[s,b]^2 + sum_a C[a,s]^2) / 2 and its square root, for the m seed strings
__global__ void k_sci_weights(const double* __restrict__ C, int m, double* __restrict__ sw) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= m) return;
    double r = 0.0, c = 0.0;
    for (int b = 0; b < m; b++) r += C[(long long)s * m + b] * C[(long long)s * m + b];
    for (int a = 0; a < m; a++) c += C[(long long)a * m + s] * C[(long long)a * m + s];
    sw[s] = sqrt(0.5 * (r + c));
}

// score of every string: max over seeds s of |H^ss_{s' s}| sqrt(w_s); seeds score +inf
__global__ void k_sci_score(SciTabs T, const unsigned* __restrict__ strs, long long nstr,
                            const unsigned* __restrict__ seed_str, const int* __restrict__ seed_map,
                            const double* __restrict__ sw, int nseed, double* __restrict__ score) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nstr) return;
    if (seed_map[i] >= 0) {
        score[i] = INFINITY;
        return;
    }
    const unsigned I = strs[i];
    double best = 0.0;
    for (int s = 0; s < nseed; s++) {
        const unsigned J = seed_str[s];
        if (__popc(I ^ J) > 4) continue;
        const double v = fabs(ss_offdiag(T, J, I)) * sw[s];
        best = fmax(best, v);
    }
    score[i] = best;
}

// the seed solution embedded in the larger product space: X[pos a][pos b] = C0[a][b]
__global__ void k_sci_embed(const double* __restrict__ C0, int m0, const int* __restrict__ seed_sel,
                            const int* __restrict__ map, int m, double* __restrict__ X) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)m0 * m0) return;
    const int a = (int)(i / m0), b = (int)(i % m0);
    const int pa = map[seed_sel[a]], pb = map[seed_sel[b]];
    if (pa >= 0 && pb >= 0) X[(long long)pa * m + pb] = C0[i];
}

// ---------------------------------------------------------------------------- reference outputs

// determinant k = a m + b: full core, alpha string a and beta string b shifted past the core
__global__ void k_sci_dets(const unsigned* __restrict__ sstr, int m, int nc, int W, unsigned long long* __restrict__ dets) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)m * m) return;
    const unsigned s[2] = {sstr[k / m], sstr[k % m]};
    for (int sp = 0; sp < 2; sp++) {
        unsigned long long w[2] = {0ull, 0ull};
        for (int i = 0; i < nc; i++) w[i >> 6] |= 1ull << (i & 63);
        for (unsigned x = s[sp]; x; x &= x - 1) {
            const int p = nc + __ffs(x) - 1;
            w[p >> 6] |= 1ull << (p & 63);
        }
        for (int q = 0; q < W; q++) dets[k * 2 * W + sp * W + q] = w[q];
    }
}

// spin-summed 1-RDM numerators: block per selected string J, entry c of its list (I, tu, s):
// s (sum_b C[J,b] C[I,b] + sum_a C[a,J] C[a,I]) into part[c m + J]
__global__ void k_sci_rdm_terms(ProdDev P, const double* __restrict__ C, double* __restrict__ part) {
    __shared__ double red[32];
    const int J = blockIdx.x, m = P.m, n = P.cnt[J];
    for (int c = 0; c < n; c++) {
        const unsigned e = P.ent[(long long)c * m + J];
        const int I = (int)(e & 0xffffu);
        double s = 0.0;
        for (int b = threadIdx.x; b < m; b += blockDim.x)
            s += C[(long long)J * m + b] * C[(long long)I * m + b] + C[(long long)b * m + J] * C[(long long)b * m + I];
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
            part[(long long)c * m + J] = (e >> 31) ? -t : t;
        }
        __syncthreads();
    }
}

// gamma[tu] = sum of the terms with that (t, u), in (c, J) order, / norm
__global__ void k_sci_rdm_sum(ProdDev P, const double* __restrict__ part, double norm, double* __restrict__ gamma) {
    const int tu = blockIdx.x * blockDim.x + threadIdx.x, m = P.m;
    if (tu >= P.na * P.na) return;
    double s = 0.0;
    for (int c = 0; c < P.cap; c++)
        for (int J = 0; J < m; J++)
            if (c < P.cnt[J] && (int)((P.ent[(long long)c * m + J] >> 16) & 0x3ffu) == tu) s += part[(long long)c * m + J];
    gamma[tu] = s / norm;
}

// generalised Fock F_pq = h_pq + sum_i [2(pq|ii) - (pi|iq)] + sum_tu gamma_tu [(pq|tu) - (pt|uq)/2]
__global__ void k_sci_fock(const double* __restrict__ h1, const double* __restrict__ eri, const double* __restrict__ gamma,
                           int n, int nc, int na, double* __restrict__ F) {
    const int pq = blockIdx.x * blockDim.x + threadIdx.x;
    if (pq >= n * n) return;
    const int p = pq / n, q = pq % n;
    double v = h1[pq];
    for (int i = 0; i < nc; i++) v += 2.0 * eri[eidx(p, q, i, i)] - eri[eidx(p, i, i, q)];
    for (int t = 0; t < na; t++)
        for (int u = 0; u < na; u++)
            v += gamma[t * na + u] * (eri[eidx(p, q, nc + t, nc + u)] - 0.5 * eri[eidx(p, nc + t, nc + u, q)]);
    F[pq] = v;
}

// ---------------------------------------------------------------------------- orbital rotation

__global__ void k_sci_unpack(const double* __restrict__ eri, int n, double* __restrict__ full) {
    const long long n2 = (long long)n * n, n4 = n2 * n2;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n4; x += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(x % n), r = (int)((x / n) % n), q = (int)((x / n2) % n), p = (int)(x / (n2 * n));
        full[x] = eri[eidx(p, q, r, s)];
    }
}

// out[s][row] = sum_{s'} U[s'][s] in[row][s'] over rows of n entries (the last index transformed
// and moved to the front); U is block diagonal, blk[s] = first index of the block of s, blk[n + s]
// = one past its last
constexpr int ROT_ROWS = 32;
__global__ void __launch_bounds__(256) k_sci_rotate(const double* __restrict__ in, long long R, int n,
                                                    const double* __restrict__ U, const int* __restrict__ blk,
                                                    double* __restrict__ out) {
    extern __shared__ double tile[];                  // ROT_ROWS x (n + 1)
    const long long row0 = (long long)blockIdx.x * ROT_ROWS;
    const int ld = n + 1;
    for (int x = threadIdx.x; x < ROT_ROWS * n; x += blockDim.x) {
        const int r = x / n, c = x % n;
        tile[r * ld + c] = row0 + r < R ? in[(row0 + r) * n + c] : 0.0;
    }
    __syncthreads();
    const int r = threadIdx.x & (ROT_ROWS - 1);
    for (int s = threadIdx.x / ROT_ROWS; s < n; s += blockDim.x / ROT_ROWS) {
        double v = 0.0;
        for (int sp = blk[s], e = blk[n + s]; sp < e; sp++) v += U[sp * n + s] * tile[r * ld + sp];
        if (row0 + r < R) out[(long long)s * R + row0 + r] = v;
    }
}

__host__ __device__ inline long long tri_root(long long x) {        // largest p with p(p+1)/2 <= x
    long long p = (long long)((sqrt(8.0 * (double)x + 1.0) - 1.0) * 0.5);
    while (p * (p + 1) / 2 > x) p--;
    while ((p + 1) * (p + 2) / 2 <= x) p++;
    return p;
}

__global__ void k_sci_pack(const double* __restrict__ full, int n, long long neri, double* __restrict__ eri) {
    const long long n2 = (long long)n * n;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < neri; x += (long long)gridDim.x * blockDim.x) {
        const long long P1 = tri_root(x), P2 = x - P1 * (P1 + 1) / 2;
        const long long p = tri_root(P1), q = P1 - p * (p + 1) / 2, r = tri_root(P2), s = P2 - r * (r + 1) / 2;
        eri[x] = full[((p * n + q) * n + r) * n + s];
        (void)n2;
    }
}

// h' = U^T h U, symmetrised
__global__ void k_sci_rot_h1(const double* __restrict__ h1, const double* __restrict__ U, const int* __restrict__ blk,
                             int n, double* __restrict__ out) {
    const int pq = blockIdx.x * blockDim.x + threadIdx.x;
    if (pq >= n * n) return;
    const int p = pq / n, q = pq % n;
    auto elem = [&](int a, int b) {
        double v = 0.0;
        for (int i = blk[a]; i < blk[n + a]; i++)
            for (int j = blk[b]; j < blk[n + b]; j++) v += U[i * n + a] * h1[i * n + j] * U[j * n + b];
        return v;
    };
    out[pq] = 0.5 * (elem(p, q) + elem(q, p));
}

}  // namespace

// ============================================================================ host driver

namespace {

struct DevBufs {                                  // device allocations of one call, freed on return
    std::vector<void*> p;
    ~DevBufs() {
        for (void* q : p) cudaFree(q);
    }
    template <class T>
    cudaError_t get(T*& out, long long n) {
        void* q = nullptr;
        const cudaError_t e = cudaMalloc(&q, sizeof(T) * (size_t)std::max(1LL, n));
        if (e == cudaSuccess) {
            p.push_back(q);
            out = (T*)q;
        }
        return e;
    }
    void drop(void* q) {
        for (auto& x : p)
            if (x == q) {
                cudaFree(x);
                x = nullptr;
            }
    }
};

// symmetric eigenproblem by cyclic Jacobi rotations: eigenvalues ascending in w, eigenvectors in the
// columns of V (row-major n x n)
void jacobi_eigh(int n, std::vector<double> A, std::vector<double>& w, std::vector<double>& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; i++) V[(size_t)i * n + i] = 1.0;
    double scale = 0.0;
    for (double a : A) scale = std::max(scale, std::fabs(a));
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0;
        for (int p = 0; p < n; p++)
            for (int q = p + 1; q < n; q++) off = std::max(off, std::fabs(A[(size_t)p * n + q]));
        if (!(off > 1e-300) || off <= 1e-17 * scale) break;
        for (int p = 0; p < n; p++)
            for (int q = p + 1; q < n; q++) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double th = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
                const double t = (th >= 0.0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; k++) {          // columns p, q: A J
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; k++) {          // rows p, q: J^T (A J)
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; k++) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    std::vector<int> ord(n);
    for (int i = 0; i < n; i++) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return A[(size_t)a * n + a] < A[(size_t)b * n + b]; });
    std::vector<double> V2((size_t)n * n);
    w.resize(n);
    for (int j = 0; j < n; j++) {
        w[j] = A[(size_t)ord[j] * n + ord[j]];
        for (int i = 0; i < n; i++) V2[(size_t)i * n + j] = V[(size_t)i * n + ord[j]];
    }
    V.swap(V2);
}

struct Space {
    int m = 0, cap = 0;
    int *sel = nullptr, *map = nullptr, *row = nullptr, *col = nullptr, *cnt = nullptr;
    unsigned *sstr = nullptr, *ent = nullptr;
    double *val = nullptr, *diag = nullptr;
    ProdDev P{};
};

struct SciRun {
    mrq_ctx* ctx;
    cudaStream_t st;
    DevBufs& buf;
    int na, ne;
    long long nstr;
    Binom B;
    SciTabs T;
    const unsigned* strs;
    const double* hd;
    const double* g;
    double ecore;
    int sms;

    int sync() {
        mrq_ctx* ctx = this->ctx;
        SCK(cudaStreamSynchronize(st));
        return 0;
    }

    // product space of the m strings whose full indices are sel (ascending)
    int build_space(int* sel, int m, Space& S) {
        mrq_ctx* ctx = this->ctx;
        S.m = m;
        S.sel = sel;
        S.cap = ne + ne * (na - ne);
        SCK(buf.get(S.map, nstr));
        SCK(buf.get(S.sstr, m));
        SCK(buf.get(S.row, m + 1));
        SCK(buf.get(S.cnt, m));
        SCK(buf.get(S.ent, (long long)S.cap * m));
        SCK(buf.get(S.diag, (long long)m * m));
        SCK(cudaMemsetAsync(S.map, 0xff, sizeof(int) * nstr, st));
        k_sci_select_map<<<(m + 255) / 256, 256, 0, st>>>(sel, m, strs, S.map, S.sstr);
        const unsigned rb = (unsigned)(((long long)m * 32 + 255) / 256);
        k_sci_rows<<<rb, 256, 0, st>>>(S.sstr, sel, m, T, hd, 0, S.row, nullptr, nullptr);
        SCK(cudaGetLastError());
        std::vector<int> row(m + 1);
        SCK(cudaMemcpyAsync(row.data(), S.row, sizeof(int) * m, cudaMemcpyDeviceToHost, st));
        if (int r = sync()) return r;
        long long run = 0;
        for (int k = 0; k < m; k++) {
            const long long c = row[k];
            row[k] = (int)run;
            run += c;
        }
        row[m] = (int)run;
        SCK(cudaMemcpyAsync(S.row, row.data(), sizeof(int) * (m + 1), cudaMemcpyHostToDevice, st));
        SCK(buf.get(S.col, run));
        SCK(buf.get(S.val, run));
        k_sci_rows<<<rb, 256, 0, st>>>(S.sstr, sel, m, T, hd, 1, S.row, S.col, S.val);
        k_sci_oslists<<<(m + 127) / 128, 128, 0, st>>>(S.sstr, m, na, ne, B, S.map, S.ent, S.cnt);
        S.P = ProdDev{m, na, S.cap, S.sstr, S.row, S.col, S.val, S.ent, S.cnt, g, ecore};
        const long long N = (long long)m * m;
        k_sci_pdiag<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(S.P, sel, hd, S.diag);
        SCK(cudaGetLastError());
        return sync();      // the host copy of the offsets must outlive the upload
    }

    int sigma(const Space& S, const double* x, double* y) {
        mrq_ctx* ctx = this->ctx;
        k_sci_sigma<<<S.m, 256, sizeof(unsigned) * std::max(1, S.cap), st>>>(S.P, x, y);
        SCK(cudaGetLastError());
        return 0;
    }

    // out[r] = A[r] . y for r < nrows (rows of length N)
    int dots(const double* A, int nrows, long long N, const double* y, double* part, double* dout, double* out) {
        mrq_ctx* ctx = this->ctx;
        k_sci_dots<<<dim3(DOT_BLOCKS, nrows), 256, 0, st>>>(A, N, y, part);
        k_sci_dots_fin<<<(nrows + 63) / 64, 64, 0, st>>>(part, DOT_BLOCKS, nrows, dout);
        SCK(cudaGetLastError());
        SCK(cudaMemcpyAsync(out, dout, sizeof(double) * nrows, cudaMemcpyDeviceToHost, st));
        return sync();
    }

    int combine(const double* A, long long N, int k, const double* c, double beta, double* out) {
        mrq_ctx* ctx = this->ctx;
        Coefs cf{};
        for (int j = 0; j < k; j++) cf.c[j] = c[j];
        k_sci_combine<<<4 * sms, 256, 0, st>>>(A, N, k, cf, beta, out);
        SCK(cudaGetLastError());
        return 0;
    }

    // lowest eigenpair of H in the product space S; x holds the start vector and receives the
    // normalised eigenvector
    int davidson(const Space& S, double* x, double tol, int max_iter, int max_sub, double& e, int& iters, double& res) {
        mrq_ctx* ctx = this->ctx;
        const long long N = (long long)S.m * S.m;
        double *V = nullptr, *AV = nullptr, *ax = nullptr, *r = nullptr, *t = nullptr, *part = nullptr, *dout = nullptr;
        SCK(buf.get(V, (long long)max_sub * N));
        SCK(buf.get(AV, (long long)max_sub * N));
        SCK(buf.get(ax, N));
        SCK(buf.get(r, N));
        SCK(buf.get(t, N));
        SCK(buf.get(part, (long long)DOT_BLOCKS * SCI_MAX_SUB));
        SCK(buf.get(dout, SCI_MAX_SUB));
        const unsigned gb = 4u * (unsigned)sms;
        std::vector<double> M((size_t)max_sub * max_sub), d(SCI_MAX_SUB), c(SCI_MAX_SUB), w, U;
        double nn = 0.0;
        if (int q = dots(x, 1, N, x, part, dout, &nn)) return q;
        if (!(nn > 0.0)) return mrq_internal_fail(ctx, MRQ_INVALID_ARG, "Davidson start vector is zero");
        SCK(cudaMemcpyAsync(V, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        k_sci_scale<<<gb, 256, 0, st>>>(V, N, 1.0 / std::sqrt(nn));
        if (int q = sigma(S, V, AV)) return q;
        if (int q = dots(V, 1, N, AV, part, dout, &M[0])) return q;
        int k = 1;
        e = M[0];
        res = INFINITY;
        iters = 0;
        for (int it = 0; it < max_iter; it++) {
            iters = it + 1;
            std::vector<double> Hs((size_t)k * k);
            for (int i = 0; i < k; i++)
                for (int j = 0; j < k; j++)
                    Hs[(size_t)i * k + j] = 0.5 * (M[(size_t)i * max_sub + j] + M[(size_t)j * max_sub + i]);
            jacobi_eigh(k, Hs, w, U);
            e = w[0];
            if (!std::isfinite(e)) return mrq_internal_fail(ctx, MRQ_CUDA_ERROR, "Davidson reached a non-finite energy");
            for (int i = 0; i < k; i++) c[i] = U[(size_t)i * k];
            if (int q = combine(V, N, k, c.data(), 0.0, x)) return q;
            if (int q = combine(AV, N, k, c.data(), 0.0, ax)) return q;
            k_sci_precond<<<gb, 256, 0, st>>>(x, ax, S.diag, e, N, r, t);
            double rr = 0.0;
            if (int q = dots(r, 1, N, r, part, dout, &rr)) return q;
            res = std::sqrt(rr);
            if (res < tol) break;
            if (k >= max_sub) {                      // restart from the current Ritz pair
                SCK(cudaMemcpyAsync(V, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
                SCK(cudaMemcpyAsync(AV, ax, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
                if (int q = dots(V, 1, N, AV, part, dout, &M[0])) return q;
                k = 1;
            }
            for (int pass = 0; pass < 2; pass++) {   // classical Gram-Schmidt, twice
                if (int q = dots(V, k, N, t, part, dout, d.data())) return q;
                for (int i = 0; i < k; i++) d[i] = -d[i];
                if (int q = combine(V, N, k, d.data(), 1.0, t)) return q;
            }
            double tt = 0.0;
            if (int q = dots(t, 1, N, t, part, dout, &tt)) return q;
            const double nt = std::sqrt(tt);
            if (nt < 1e-14) break;
            double* vk = V + (long long)k * N;
            double* avk = AV + (long long)k * N;
            SCK(cudaMemcpyAsync(vk, t, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
            k_sci_scale<<<gb, 256, 0, st>>>(vk, N, 1.0 / nt);
            if (int q = sigma(S, vk, avk)) return q;
            if (int q = dots(V, k + 1, N, avk, part, dout, d.data())) return q;     // V_i . AV_k
            for (int i = 0; i <= k; i++) M[(size_t)i * max_sub + k] = d[i];
            if (int q = dots(AV, k, N, vk, part, dout, d.data())) return q;         // V_k . AV_i
            for (int i = 0; i < k; i++) M[(size_t)k * max_sub + i] = d[i];
            k++;
        }
        double xx = 0.0;
        if (int q = dots(x, 1, N, x, part, dout, &xx)) return q;
        k_sci_scale<<<gb, 256, 0, st>>>(x, N, 1.0 / std::sqrt(xx));
        SCK(cudaGetLastError());
        if (int q = sync()) return q;
        buf.drop(V);
        buf.drop(AV);
        return 0;
    }
};

}  // namespace

extern "C" int mrq_sci_reference(mrq_ctx* ctx, const mrq_sci_params* p, mrq_sci_result* out, uint32_t* strings_out,
                                 double* coeffs_out) {
    if (!ctx) return MRQ_INVALID_ARG;
    if (!p || !out) return mrq_internal_fail(ctx, MRQ_INVALID_ARG, "null parameters or result");
    MrqHamView H{};
    if (int r = mrq_internal_ham(ctx, &H)) return r;
    const auto t0 = std::chrono::steady_clock::now();
    if (H.nalpha != H.nbeta)
        return mrq_internal_fail(ctx, MRQ_INVALID_ARG, "the selected-CI reference is built for Sz = 0 (n_alpha = n_beta)");
    const int na = H.na, ne = H.nalpha - H.nc;
    if (na < 1) return mrq_internal_fail(ctx, MRQ_INVALID_ARG, "no active orbitals");
    Binom B{};
    for (int i = 0; i <= 32; i++) {
        B.c[i][0] = 1;
        for (int j = 1; j <= i; j++) B.c[i][j] = B.c[i - 1][j - 1] + (j <= i - 1 ? B.c[i - 1][j] : 0);
    }
    const long long nstr = (long long)B.c[na][ne];
    if (nstr > SCI_MAX_SPACE)
        return mrq_internal_fail(ctx, MRQ_TOO_LARGE, "%lld strings of %d electrons in %d orbitals (at most %lld)", nstr,
                                 ne, na, SCI_MAX_SPACE);
    const int nseed = (int)std::min<long long>(p->n_seed_strings, nstr);
    const int nsel = (int)std::min<long long>(p->n_strings, nstr);
    if (nseed < 1 || nsel < nseed || nsel > SCI_MAX_STR)
        return mrq_internal_fail(ctx, MRQ_INVALID_ARG, "need 1 <= n_seed_strings <= n_strings <= %d", SCI_MAX_STR);
    if (!(p->tol > 0.0) || p->max_iter < 1 || p->max_sub < 2 || p->max_sub > SCI_MAX_SUB)
        return mrq_internal_fail(ctx, MRQ_INVALID_ARG, "need tol > 0, max_iter >= 1, 2 <= max_sub <= %d", SCI_MAX_SUB);
    SCK(cudaSetDevice(H.device));
    if (int r = mrq_internal_sync(ctx)) return r;
    cudaStream_t st = H.stream;
    int sms = 0;
    SCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, H.device));
    DevBufs buf;
    const int n = H.n, nc = H.nc;
    const long long na2 = (long long)na * na;
    double *g = nullptr, *h = nullptr, *d_ecore = nullptr, *hd = nullptr;
    unsigned* strs = nullptr;
    SCK(buf.get(g, na2 * na2));
    SCK(buf.get(h, na2));
    SCK(buf.get(d_ecore, 1));
    SCK(buf.get(strs, nstr));
    SCK(buf.get(hd, nstr));
    k_sci_active<<<std::max(1, (int)std::min<long long>(4LL * sms, (na2 * na2 + na2 + 256) / 256)), 256, 0, st>>>(
        H.h1, H.eri, n, nc, na, H.e_nuc, g, h, d_ecore);
    k_sci_unrank<<<(unsigned)((nstr + 255) / 256), 256, 0, st>>>(B, na, ne, nstr, strs);
    SciTabs T{g, h, na};
    k_sci_diag<<<(unsigned)((nstr + 255) / 256), 256, 0, st>>>(T, strs, nstr, hd);
    SCK(cudaGetLastError());
    double ecore = 0.0;
    SCK(cudaMemcpyAsync(&ecore, d_ecore, sizeof(double), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    SciRun R{ctx, st, buf, na, ne, nstr, B, T, strs, hd, g, ecore, sms};

    // seed strings: the nseed lowest one-spin energies (first on ties)
    unsigned char* flag = nullptr;
    int *seed_sel = nullptr, *sel = nullptr, *d_count = nullptr;
    long long* d_idx = nullptr;
    SCK(buf.get(flag, nstr));
    SCK(buf.get(seed_sel, nseed));
    SCK(buf.get(sel, nsel));
    SCK(buf.get(d_count, 1));
    SCK(buf.get(d_idx, 1));
    const unsigned rbl = (unsigned)((nstr + 255) / 256);
    k_sci_rank_select<<<rbl, 256, 256 * sizeof(double), st>>>(hd, nstr, nseed, 0, flag);
    k_sci_compact<<<1, 1024, 0, st>>>(flag, nstr, seed_sel, nseed, d_count);
    SCK(cudaGetLastError());
    int count = 0;
    SCK(cudaMemcpyAsync(&count, d_count, sizeof(int), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    if (count != nseed) return mrq_internal_fail(ctx, MRQ_CUDA_ERROR, "seed selection found %d strings", count);
    Space S0;
    if (int r = R.build_space(seed_sel, nseed, S0)) return r;
    const long long N0 = (long long)nseed * nseed;
    double* C0 = nullptr;
    SCK(buf.get(C0, N0));
    SCK(cudaMemsetAsync(C0, 0, sizeof(double) * N0, st));
    long long imin = 0;
    k_sci_argext<<<1, 1024, 0, st>>>(S0.diag, N0, 0, d_idx);
    SCK(cudaMemcpyAsync(&imin, d_idx, sizeof(long long), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    const double one = 1.0;
    SCK(cudaMemcpyAsync(C0 + imin, &one, sizeof(double), cudaMemcpyHostToDevice, st));
    k_sci_noise<<<4 * sms, 256, 0, st>>>(C0, N0, 11ull);
    double e_seed = 0.0, res0 = 0.0;
    int it0 = 0;
    if (int r = R.davidson(S0, C0, p->tol, p->max_iter, p->max_sub, e_seed, it0, res0)) return r;

    // heat-bath scores against the seed solution; the nsel best strings (seeds first, then by score,
    // first on ties)
    double *sw = nullptr, *score = nullptr;
    SCK(buf.get(sw, nseed));
    SCK(buf.get(score, nstr));
    k_sci_weights<<<(nseed + 127) / 128, 128, 0, st>>>(C0, nseed, sw);
    k_sci_score<<<rbl, 256, 0, st>>>(T, strs, nstr, S0.sstr, S0.map, sw, nseed, score);
    k_sci_rank_select<<<rbl, 256, 256 * sizeof(double), st>>>(score, nstr, nsel, 1, flag);
    k_sci_compact<<<1, 1024, 0, st>>>(flag, nstr, sel, nsel, d_count);
    SCK(cudaGetLastError());
    SCK(cudaMemcpyAsync(&count, d_count, sizeof(int), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    if (count != nsel)
        return mrq_internal_fail(ctx, MRQ_CUDA_ERROR, "selection found %d strings (scores not finite?)", count);
    Space S1;
    if (int r = R.build_space(sel, nsel, S1)) return r;
    const long long N1 = (long long)nsel * nsel;
    double* C = nullptr;
    SCK(buf.get(C, N1));
    SCK(cudaMemsetAsync(C, 0, sizeof(double) * N1, st));
    k_sci_embed<<<(unsigned)((N0 + 255) / 256), 256, 0, st>>>(C0, nseed, seed_sel, S1.map, nsel, C);
    k_sci_noise<<<4 * sms, 256, 0, st>>>(C, N1, 11ull);
    double e = 0.0, res = 0.0;
    int it1 = 0;
    if (int r = R.davidson(S1, C, p->tol, p->max_iter, p->max_sub, e, it1, res)) return r;
    k_sci_argext<<<1, 1024, 0, st>>>(C, N1, 1, d_idx);
    long long imax = 0;
    double cmax = 0.0;
    SCK(cudaMemcpyAsync(&imax, d_idx, sizeof(long long), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    SCK(cudaMemcpyAsync(&cmax, C + imax, sizeof(double), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    if (cmax < 0.0) k_sci_scale<<<4 * sms, 256, 0, st>>>(C, N1, -1.0);

    // semicanonical core and virtual orbitals: diagonalise F_cc and F_vv with the reference's
    // spin-summed 1-RDM, rotate h1 and (pq|rs), reload the Hamiltonian
    double fock_off = 0.0;
    if (p->semicanonical) {
        double *part = nullptr, *gamma = nullptr, *F = nullptr;
        SCK(buf.get(part, (long long)std::max(1, S1.cap) * nsel));
        SCK(buf.get(gamma, na2));
        SCK(buf.get(F, (long long)n * n));
        SCK(cudaMemsetAsync(part, 0, sizeof(double) * std::max(1, S1.cap) * nsel, st));
        k_sci_rdm_terms<<<nsel, 256, 0, st>>>(S1.P, C, part);
        k_sci_rdm_sum<<<(unsigned)((na2 + 63) / 64), 64, 0, st>>>(S1.P, part, 1.0, gamma);
        k_sci_fock<<<(n * n + 127) / 128, 128, 0, st>>>(H.h1, H.eri, gamma, n, nc, na, F);
        SCK(cudaGetLastError());
        std::vector<double> Fh((size_t)n * n), U((size_t)n * n, 0.0);
        std::vector<int> blk(2 * n);
        SCK(cudaMemcpyAsync(Fh.data(), F, sizeof(double) * n * n, cudaMemcpyDeviceToHost, st));
        SCK(cudaStreamSynchronize(st));
        for (int q = 0; q < n; q++) U[(size_t)q * n + q] = 1.0;
        const int lo[3] = {0, nc, nc + na}, hi[3] = {nc, nc + na, n};
        for (int b = 0; b < 3; b++) {
            for (int q = lo[b]; q < hi[b]; q++) {
                blk[q] = b == 1 ? q : lo[b];
                blk[n + q] = b == 1 ? q + 1 : hi[b];
            }
            if (b == 1 || hi[b] == lo[b]) continue;
            const int k = hi[b] - lo[b];
            std::vector<double> A((size_t)k * k), w, V;
            for (int i = 0; i < k; i++)
                for (int j = 0; j < k; j++) {
                    A[(size_t)i * k + j] = 0.5 * (Fh[(size_t)(lo[b] + i) * n + lo[b] + j] + Fh[(size_t)(lo[b] + j) * n + lo[b] + i]);
                    if (i != j) fock_off = std::max(fock_off, std::fabs(Fh[(size_t)(lo[b] + i) * n + lo[b] + j]));
                }
            jacobi_eigh(k, A, w, V);
            for (int i = 0; i < k; i++)
                for (int j = 0; j < k; j++) U[(size_t)(lo[b] + i) * n + lo[b] + j] = V[(size_t)i * k + j];
        }
        double *dU = nullptr, *h1r = nullptr, *erir = nullptr, *X = nullptr, *Y = nullptr;
        int* dblk = nullptr;
        const long long n4 = (long long)n * n * n * n, R3 = (long long)n * n * n;
        SCK(buf.get(dU, (long long)n * n));
        SCK(buf.get(dblk, 2LL * n));
        SCK(buf.get(h1r, (long long)n * n));
        SCK(buf.get(erir, H.neri));
        SCK(buf.get(X, n4));
        SCK(buf.get(Y, n4));
        SCK(cudaMemcpyAsync(dU, U.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice, st));
        SCK(cudaMemcpyAsync(dblk, blk.data(), sizeof(int) * 2 * n, cudaMemcpyHostToDevice, st));
        k_sci_rot_h1<<<(n * n + 127) / 128, 128, 0, st>>>(H.h1, dU, dblk, n, h1r);
        k_sci_unpack<<<8 * sms, 256, 0, st>>>(H.eri, n, X);
        const size_t rsm = sizeof(double) * ROT_ROWS * (n + 1);
        for (int pass = 0; pass < 4; pass++) {
            k_sci_rotate<<<(unsigned)((R3 + ROT_ROWS - 1) / ROT_ROWS), 256, rsm, st>>>(X, R3, n, dU, dblk, Y);
            std::swap(X, Y);
        }
        k_sci_pack<<<8 * sms, 256, 0, st>>>(X, n, H.neri, erir);
        SCK(cudaGetLastError());
        SCK(cudaStreamSynchronize(st));
        buf.drop(X);
        buf.drop(Y);
        if (int r = mrq_load_hamiltonian(ctx, nc, na, H.nv, H.nalpha, H.nbeta, h1r, erir, H.e_nuc)) return r;
    }

    // the reference: n_strings^2 determinants and their coefficients, loaded as mrq_load_reference does
    unsigned long long* dets = nullptr;
    SCK(buf.get(dets, N1 * 2 * H.W));
    k_sci_dets<<<(unsigned)((N1 + 255) / 256), 256, 0, st>>>(S1.sstr, nsel, nc, H.W, dets);
    SCK(cudaGetLastError());
    SCK(cudaStreamSynchronize(st));
    if (int r = mrq_load_reference(ctx, N1, (const uint64_t*)dets, C)) return r;
    if (strings_out) SCK(cudaMemcpy(strings_out, S1.sstr, sizeof(unsigned) * nsel, cudaMemcpyDefault));
    if (coeffs_out) SCK(cudaMemcpy(coeffs_out, C, sizeof(double) * N1, cudaMemcpyDefault));
    out->energy = e;
    out->seed_energy = e_seed;
    out->residual = res;
    out->fock_offdiag = fock_off;
    out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    out->n_det = N1;
    out->n_strings = nsel;
    out->n_seed_strings = nseed;
    out->iters_seed = it0;
    out->iters = it1;
    return 0;
}
