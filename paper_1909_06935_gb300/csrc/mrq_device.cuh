// Device-side building blocks of the local-estimator path (sm_103a, FP64).
//
//  - determinant bit operations on W uint64 words per spin string,
//  - packed two-electron integral gathers,
//  - Slater-Condon matrix elements of H and of Dyall's H_D (Sec. II C),
//  - perturber labels (Sec. II A, spin-orbital reading),
//  - the reference hash table (Sec. II D: "stored in a hash table ... constant time"),
//  - reach-back overlaps O(m) = <m|H|phi0> (Eq. 6-7, Sec. II D second layer),
//  - Philox4x32-10 (Salmon et al., SC'11) for the first-reaction move selection.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define MRQ_MAXN 128
#define MRQ_MAXB 171
#define MRQ_EMPTY_KEY 0xFFFFFFFFFFFFFFFFull

// device error flags (OR-ed into SysDev::err)
#define MRQ_ERR_HASH 1
#define MRQ_ERR_NOMOVE 2
#define MRQ_ERR_LABEL 4
#define MRQ_ERR_CAP 64          // a candidate list outgrew its shared-memory capacity

struct HashSlot {
    unsigned long long key;
    double val;
};

// Everything a kernel needs to know about one loaded system.  Lives in device memory; the
// batched launcher keeps an array of these and walkers carry an index into it.
struct SysDev {
    int n, nc, na, nv, W;
    int nalpha, nbeta;
    long long nPs, nlab;
    unsigned long long mcore[2], mact[2], mvirt[2];   // orbital masks per word (same for both spins)
    const double* eri;      // packed (input layout)
    const double* eri4;     // half-unpacked: E[P(p,q)][r][s] = (pq|rs), n(n+1)/2 x n x n
    // physicists' tables over the blocks the CAS path reads: p, q in core+active (nca), r, s in
    // active+virtual (nav, index minus n_core): T[p][q][r][s] = <pq|rs> = (pr|qs), then, after
    // tab_half entries, <pq||rs> = (pr|qs) - (ps|qr)
    const double* tab;
    int nca, nav;
    unsigned tab_half;
    const double* hc;       // n*n: h_pq + sum_i [2(pq|ii) - (pi|iq)] (full core)
    const double* h1;       // n*n
    const double* eps;      // n: generalised-Fock diagonal
    double e_nuc, e_core, e0, sum_eps_core;
    const HashSlot* hash;
    unsigned long long hmask;
    int max_probe;
    int cand_cap;           // per-warp candidate-list capacity (shared memory) of the CAS path
    const double* c;        // nlab sampling coefficients
    // accumulators (G groups)
    double* accN;
    double* accU;
    double* accW;
    double* accE;
    double* accA;           // [G][nlab] sum w E_L / c_l      (SC-MRCI gradient, Eq. 8-9)
    double* accB;           // [G][nlab] sum w / c_l
    unsigned long long* type_steps;
    int G;
    long long burn_in;
    unsigned long long seed;
    int* err;
    // work-unit plan of a CAS walker's step (the same for every CAS determinant of the system:
    // they all hold the same numbers of active alpha and beta electrons)
    long long cas_nb_total;  // neighbours of a CAS determinant
    int cas_nb;              // of them inside the CAS
    int cas_units;           // units covering those (MRQ_CAS_CH each)
    int unit_off[9];         // first unit of pair class k = 3 ka + kb (k < 8); unit_off[8] = all units
    int nch[8];              // chunks per (X_a, Y_a) pair of class k
    int gstride;             // doubles of the walker's single-excitation operator, 2 nca nav
    int hb_on;               // heat-bath cutoff in force (hb_eps > 0)
    const unsigned short* colex;       // pair decode table: colex[j(j-1)/2 + i] = i | j << 8, i < j < 128
    unsigned long long mag_c, mag_v;   // ceil(2^64 / n_core), ceil(2^64 / n_virt) (0 when that is <= 1)
    double hb_eps;           // heat-bath cutoff: double excitations with |<ab||ij>| < hb_eps are dropped
};

// The heat-bath cutoff (Sec. II D generates excitations by the heat-bath algorithm; with a
// positive cutoff it drops every double excitation whose element |<ab||ij>| is below it): the walk's
// double-excitation elements pass through this screen.  Off (no FP64 compare) at cutoff zero.
__device__ __forceinline__ double hb_screen(const SysDev& S, double v) {
    if (S.hb_on && fabs(v) < S.hb_eps) v = 0.0;
    return v;
}

// ------------------------------------------------------------------ access counters
// The walk uses NoCtr (compiles away); the parity/debug kernel uses Ctr to report, per
// determinant, the random global accesses the algorithm makes (integral and table gathers,
// hash-slot reads) and the reach-back candidates it tries.
struct NoCtr {
    __device__ __forceinline__ void g(int = 1) {}
    __device__ __forceinline__ void pr(int = 1) {}
    __device__ __forceinline__ void cand() {}
    __device__ __forceinline__ void term(int = 1) {}
    __device__ __forceinline__ void mark(int) {}     // phase boundary (timing builds only)
};
struct Ctr {
    unsigned long long gathers = 0, probes = 0, cands = 0, terms = 0;
    __device__ __forceinline__ void g(int k = 1) { gathers += k; }
    __device__ __forceinline__ void pr(int k = 1) { probes += k; }
    __device__ __forceinline__ void cand() { cands++; }
    __device__ __forceinline__ void term(int k = 1) { terms += k; }   // H_mk phi0(k) products summed
    __device__ __forceinline__ void mark(int) {}
};

// ------------------------------------------------------------------ small helpers

__device__ __forceinline__ long long pair_idx(int p, int q) {
    return p >= q ? (long long)p * (p + 1) / 2 + q : (long long)q * (q + 1) / 2 + p;
}

// (pq|rs) from the half-unpacked table, arranged by the 8-fold symmetry so that the largest
// orbital index comes last.  Lanes of a warp usually differ only in a virtual (largest) index,
// so their gathers land on consecutive addresses.  n <= 128 keeps the index below 2^31.
__device__ __forceinline__ double eri_g(const SysDev& S, int p, int q, int r, int s) {
    int m1 = p > q ? p : q, m2 = r > s ? r : s;
    if (m1 > m2) {
        int t = p; p = r; r = t;
        t = q; q = s; s = t;
    }
    if (r > s) { int t = r; r = s; s = t; }
    const unsigned P = p >= q ? (unsigned)(p * (p + 1) / 2 + q) : (unsigned)(q * (q + 1) / 2 + p);
    return __ldg(S.eri4 + (P * (unsigned)S.n + (unsigned)r) * (unsigned)S.n + (unsigned)s);
}

// index of (pq|rs) in the half-unpacked table (same arrangement as eri_g)
__device__ __forceinline__ unsigned eri_idx(const SysDev& S, int p, int q, int r, int s) {
    int m1 = p > q ? p : q, m2 = r > s ? r : s;
    if (m1 > m2) {
        int t = p; p = r; r = t;
        t = q; q = s; s = t;
    }
    if (r > s) { int t = r; r = s; s = t; }
    const unsigned P = p >= q ? (unsigned)(p * (p + 1) / 2 + q) : (unsigned)(q * (q + 1) / 2 + p);
    return (P * (unsigned)S.n + (unsigned)r) * (unsigned)S.n + (unsigned)s;
}

// number of set bits of string s strictly between orbitals lo < hi
template <int W>
__device__ __forceinline__ int popc_between(const unsigned long long* s, int lo, int hi) {
    int c = 0;
#pragma unroll
    for (int w = 0; w < W; w++) {
        int b0 = 64 * w;
        int from = lo + 1 > b0 ? lo + 1 : b0;
        int to = hi < b0 + 64 ? hi : b0 + 64;
        if (from < to) {
            int f = from - b0, t = to - b0;
            unsigned long long m = (t >= 64 ? ~0ull : ((1ull << t) - 1ull)) & ~((1ull << f) - 1ull);
            c += __popcll(s[w] & m);
        }
    }
    return c;
}

template <int W>
__device__ __forceinline__ int sgn_single(const unsigned long long* s, int p, int q) {
    int lo = p < q ? p : q, hi = p < q ? q : p;
    return (popc_between<W>(s, lo, hi) & 1) ? -1 : 1;
}

// popc_between / sgn_single on spin string sg of a determinant (row chosen by selects)
template <int W>
__device__ __forceinline__ int popc_sel(const unsigned long long (&d)[2][W], int sg, int lo, int hi) {
    unsigned long long r[W];
#pragma unroll
    for (int w = 0; w < W; w++) r[w] = sg ? d[1][w] : d[0][w];
    return popc_between<W>(r, lo, hi);
}

template <int W>
__device__ __forceinline__ int sgn_sel(const unsigned long long (&d)[2][W], int sg, int p, int q) {
    return (popc_sel<W>(d, sg, p < q ? p : q, p < q ? q : p) & 1) ? -1 : 1;
}

template <int W>
__device__ __forceinline__ bool bit_of(const unsigned long long* s, int p) {
    return (s[p >> 6] >> (p & 63)) & 1ull;
}
template <int W>
__device__ __forceinline__ void flip(unsigned long long* s, int p) {
    const unsigned long long b = 1ull << (p & 63);
    if (W == 1) {
        s[0] ^= b;
    } else {
#pragma unroll
        for (int w = 0; w < W; w++) s[w] ^= (p >> 6) == w ? b : 0ull;   // word chosen by selects, not an index
    }
}

// the same on spin string sg of a determinant, with every array index known at compile time so
// that the determinant stays in registers (a runtime row index would put it in local memory)
template <int W>
__device__ __forceinline__ void flip_reg(unsigned long long (&m)[2][W], int sg, int p) {
    const unsigned long long b = 1ull << (p & 63);
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int w = 0; w < W; w++) m[s][w] ^= (s == sg && (W == 1 || (p >> 6) == w)) ? b : 0ull;
}

// active bits of a spin string, right-aligned (n_act <= 32; the active block may straddle a word)
template <int W>
__device__ __forceinline__ unsigned active_bits(const SysDev& S, const unsigned long long* s) {
    unsigned long long v = 0;
    int lo = S.nc;
    if (W == 1) {
        v = s[0] >> lo;
    } else {
        int w = lo >> 6, b = lo & 63;
        v = s[w] >> b;
        if (b && w + 1 < W) v |= s[w + 1] << (64 - b);
    }
    return (unsigned)(v & ((S.na >= 32) ? 0xFFFFFFFFull : ((1ull << S.na) - 1ull)));
}

__device__ __forceinline__ unsigned long long hash_key(const SysDev& S, unsigned aa, unsigned ab) {
    return (unsigned long long)aa | ((unsigned long long)ab << S.na);
}

// SplitMix64 finalizer (Steele, Lea, Flood, OOPSLA 2014) as the table's hash function
__device__ __host__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

template <class C = NoCtr>
__device__ __forceinline__ double hash_lookup(const SysDev& S, unsigned long long key, C& ctr) {
    unsigned long long h = mix64(key) & S.hmask;
    for (int i = 0; i < S.max_probe; i++) {
        ctr.pr();
        const double2 e = __ldg(reinterpret_cast<const double2*>(S.hash + h));
        unsigned long long k = (unsigned long long)__double_as_longlong(e.x);
        if (k == key) return e.y;
        if (k == MRQ_EMPTY_KEY) return 0.0;
        h = (h + 1) & S.hmask;
    }
    atomicOr(S.err, MRQ_ERR_HASH);
    return 0.0;
}
__device__ __forceinline__ double hash_lookup(const SysDev& S, unsigned long long key) {
    NoCtr c;
    return hash_lookup(S, key, c);
}


// ------------------------------------------------------------------ labels

__device__ __forceinline__ long long set_rank(int cnt, int x0, int x1, int m) {
    if (cnt == 0) return 0;
    if (cnt == 1) return 1 + x0;
    return 1 + m + (long long)x1 * (x1 - 1) / 2 + x0;   // x0 < x1
}

// label and (h, p) of a determinant; label -1 outside CAS+FOIS
template <int W>
__device__ __forceinline__ long long det_label(const SysDev& S, const unsigned long long (&d)[2][W], int& h,
                                               int& p) {
    int hs[2] = {0, 0}, ps[2] = {0, 0};
    h = 0;
    p = 0;
#pragma unroll
    for (int sg = 0; sg < 2; sg++) {
        unsigned long long hm = ~d[sg][0] & S.mcore[0];     // core is in word 0 (n_core <= 64)
        while (hm) {
            int i = __ffsll(hm) - 1;
            hm &= hm - 1;
            if (h < 2) hs[h] = sg * S.nc + i;
            h++;
        }
    }
#pragma unroll
    for (int sg = 0; sg < 2; sg++)
#pragma unroll
        for (int w = 0; w < W; w++) {
            unsigned long long pm = d[sg][w] & S.mvirt[w];
            while (pm) {
                int a = 64 * w + __ffsll(pm) - 1 - S.nc - S.na;
                pm &= pm - 1;
                if (p < 2) ps[p] = sg * S.nv + a;
                p++;
            }
        }
    if (h > 2 || p > 2) return -1;
    return set_rank(h, hs[0], hs[1], 2 * S.nc) * S.nPs + set_rank(p, ps[0], ps[1], 2 * S.nv);
}

// ------------------------------------------------------------------ Slater-Condon

// <d'|H|d> for the single x -> y (spin orbitals so = sigma*n + p, same spin) applied to d:
// sign * (hc_yx + sum over occupied active/virtual j [(yx|jj) - d_ss (yj|jx)]
//               - sum over core holes j [(yx|jj) - d_ss (yj|jx)])
template <int W, class C = NoCtr>
__device__ double single_elem(const SysDev& S, const unsigned long long (&d)[2][W], int x, int y, C& ctr) {
    const int n = S.n;
    const int sx = x >= n, px = x - sx * n, py = y - sx * n;
    ctr.g();
    double v = __ldg(S.hc + py * n + px);
#pragma unroll
    for (int sg = 0; sg < 2; sg++) {
#pragma unroll
        for (int w = 0; w < W; w++) {
            unsigned long long om = d[sg][w] & (S.mact[w] | S.mvirt[w]);
            while (om) {
                int j = 64 * w + __ffsll(om) - 1;
                om &= om - 1;
                v += eri_g(S, py, px, j, j);
                ctr.g();
                if (sg == sx) { v -= eri_g(S, py, j, j, px); ctr.g(); }
            }
        }
        unsigned long long hm = ~d[sg][0] & S.mcore[0];
        while (hm) {
            int j = __ffsll(hm) - 1;
            hm &= hm - 1;
            v -= eri_g(S, py, px, j, j);
            ctr.g();
            if (sg == sx) { v += eri_g(S, py, j, j, px); ctr.g(); }
        }
    }
    return __longlong_as_double(__double_as_longlong(v) ^ ((long long)(popc_sel<W>(d, sx, px < py ? px : py, px < py ? py : px) & 1) << 63));
}

// <d'|H|d> for the double r1,r2 -> a1,a2 (spin orbitals, r1<r2, a1<a2, spin conserving)
template <int W, class C = NoCtr>
__device__ __forceinline__ double double_elem(const SysDev& S, const unsigned long long (&d)[2][W], int r1, int r2,
                                              int a1, int a2, C& ctr) {
    const int n = S.n;
    int s_r1 = r1 >= n, s_r2 = r2 >= n, s_a1 = a1 >= n, s_a2 = a2 >= n;
    int pr1 = r1 - s_r1 * n, pr2 = r2 - s_r2 * n, pa1 = a1 - s_a1 * n, pa2 = a2 - s_a2 * n;
    // pairing r1->a1, r2->a2 (spin conserving by the ordering of spin orbitals)
    int c1 = popc_sel<W>(d, s_r1, pr1 < pa1 ? pr1 : pa1, pr1 < pa1 ? pa1 : pr1);
    int c2;
    if (s_r2 == s_r1) {
        unsigned long long t[W];
#pragma unroll
        for (int w = 0; w < W; w++) t[w] = s_r1 ? d[1][w] : d[0][w];
        flip<W>(t, pr1);
        flip<W>(t, pa1);
        c2 = popc_between<W>(t, pr2 < pa2 ? pr2 : pa2, pr2 < pa2 ? pa2 : pr2);
    } else {
        c2 = popc_sel<W>(d, s_r2, pr2 < pa2 ? pr2 : pa2, pr2 < pa2 ? pa2 : pr2);
    }
    double v = eri_g(S, pa1, pr1, pa2, pr2);
    ctr.g();
    if (s_r1 == s_r2) { v -= eri_g(S, pa1, pr2, pa2, pr1); ctr.g(); }
    return ((c1 + c2) & 1) ? -v : v;
}

// <d'|H_D|d> for an active single t -> u on a determinant (Dyall: heff + active two-electron)
template <int W, class C = NoCtr>
__device__ double hd_single_elem(const SysDev& S, const unsigned long long (&d)[2][W], int x, int y, C& ctr) {
    const int n = S.n;
    const int sx = x >= n, px = x - sx * n, py = y - sx * n;
    ctr.g();
    double v = __ldg(S.hc + py * n + px);   // heff_tu = hc on the active block
#pragma unroll
    for (int sg = 0; sg < 2; sg++)
#pragma unroll
        for (int w = 0; w < W; w++) {
            unsigned long long om = d[sg][w] & S.mact[w];
            while (om) {
                int j = 64 * w + __ffsll(om) - 1;
                om &= om - 1;
                v += eri_g(S, py, px, j, j);
                ctr.g();
                if (sg == sx) { v -= eri_g(S, py, j, j, px); ctr.g(); }
            }
        }
    return __longlong_as_double(__double_as_longlong(v) ^ ((long long)(popc_sel<W>(d, sx, px < py ? px : py, px < py ? py : px) & 1) << 63));
}

// ------------------------------------------------------------------ reach-back (Eq. 6-7)
//
// O(m) = <m|H|phi0> for m outside the CAS.  A reference determinant k has a full core and empty
// virtuals, so the excitation m -> k removes every virtual electron of m (plus active electrons)
// and fills every core hole (plus active holes): R = P u R', A = H u A', |R| = |A| <= 2.

// `self_key`/`self_term`: when the walker n is itself a CAS determinant, the candidate k = n
// needs no lookup: its term is H_nm phi0(n), both already known (pass self_key = ~0 otherwise).
// Single elements from a walker's operator: <k|H|m> for the single x -> y of m (x in active +
// virtual, y in core + active, not both active) is G_yx(m) = h_yx + sum_{j in m} [(yx|jj) - delta
// (yj|jx)], taken as the walker n's G_yx(n) (g, in shared memory) plus the terms of the <= 4 spin
// orbitals in which m differs from n (removed rm*, added ad*; r of each), with m's sign.
struct SglFromWalker {
    const double* g;        // nullptr: full Slater-Condon sums
    int r, rm0, rm1, ad0, ad1;   // r = 0: m is the walker itself
};

// whether the single x -> y lies in the block the walker's operator holds
__device__ __forceinline__ bool in_walker_block(const SysDev& S, int x, int y) {
    const int sx = x >= S.n, px = x - sx * S.n, py = y - sx * S.n;
    return px >= S.nc && py < S.nca && !(py >= S.nc && px < S.nca);
}

__device__ __forceinline__ double g_corr(const SysDev& S, int sx, int px, int py, int j) {
    const int sj = j >= S.n, pj = j - sj * S.n;
    double v = eri_g(S, py, px, pj, pj);
    if (sj == sx) v -= eri_g(S, py, pj, pj, px);
    return v;
}

template <int W, class C>
__device__ __forceinline__ double single_from_walker(const SysDev& S, const SglFromWalker& G,
                                                     const unsigned long long (&m)[2][W], int x, int y, C& ctr) {
    const int sx = x >= S.n, px = x - sx * S.n, py = y - sx * S.n;
    double v = G.g[(sx * S.nca + py) * S.nav + (px - S.nc)];
    if (G.r >= 1) v += g_corr(S, sx, px, py, G.ad0) - g_corr(S, sx, px, py, G.rm0);
    if (G.r == 2) v += g_corr(S, sx, px, py, G.ad1) - g_corr(S, sx, px, py, G.rm1);
    ctr.g(1 + 4 * G.r);
    return __longlong_as_double(__double_as_longlong(v) ^ ((long long)(popc_sel<W>(m, sx, px < py ? px : py, px < py ? py : px) & 1) << 63));
}

template <int W, class C = NoCtr>
__device__ double reach_back(const SysDev& S, const unsigned long long (&m)[2][W], C& ctr,
                             unsigned long long self_key = MRQ_EMPTY_KEY, double self_term = 0.0,
                             const SglFromWalker& G = SglFromWalker{nullptr, 0, 0, 0, 0, 0}) {
    const int n = S.n, nc = S.nc, na = S.na;
    int hs[2], ps[2], hc = 0, pc = 0;
#pragma unroll
    for (int sg = 0; sg < 2; sg++) {
        unsigned long long hm = ~m[sg][0] & S.mcore[0];
        while (hm) {
            int i = __ffsll(hm) - 1;
            hm &= hm - 1;
            if (hc < 2) hs[hc] = sg * n + i;
            hc++;
        }
#pragma unroll
        for (int w = 0; w < W; w++) {
            unsigned long long pm = m[sg][w] & S.mvirt[w];
            while (pm) {
                int a = 64 * w + __ffsll(pm) - 1;
                pm &= pm - 1;
                if (pc < 2) ps[pc] = sg * n + a;
                pc++;
            }
        }
    }
    const unsigned ao0 = active_bits<W>(S, m[0]), ao1 = active_bits<W>(S, m[1]);
    const unsigned amask = (na >= 32) ? 0xFFFFFFFFu : ((1u << na) - 1u);
    const unsigned ae0 = ~ao0 & amask, ae1 = ~ao1 & amask;
    // combined active masks: alpha in bits 0..31, beta in 32..63
    const unsigned long long AO = (unsigned long long)ao0 | ((unsigned long long)ao1 << 32);
    const unsigned long long AE = (unsigned long long)ae0 | ((unsigned long long)ae1 << 32);
    int pa = 0, ha = 0;   // alpha counts among P and H
    for (int i = 0; i < pc; i++) pa += ps[i] < n;
    for (int i = 0; i < hc; i++) ha += hs[i] < n;
    double acc = 0.0;

    // r = 1
    if (hc <= 1 && pc <= 1) {
        unsigned long long Rset = pc ? 0ull : AO;     // candidates for the removed electron
        unsigned long long Aset = hc ? 0ull : AE;
        int nR = pc ? 1 : __popcll(Rset);
        for (int ir = 0; ir < nR; ir++) {
            int x, xbit = -1;
            if (pc) {
                x = ps[0];
            } else {
                xbit = __ffsll(Rset) - 1;
                Rset &= Rset - 1;
                x = (xbit >= 32 ? n : 0) + nc + (xbit & 31);
            }
            int sx = x >= n;
            unsigned long long Ac = hc ? 0ull : (Aset & (sx ? 0xFFFFFFFF00000000ull : 0xFFFFFFFFull));
            int nA = hc ? 1 : __popcll(Ac);
            for (int ia = 0; ia < nA; ia++) {
                int y, ybit = -1;
                if (hc) {
                    y = hs[0];
                    if ((y >= n) != sx) continue;
                } else {
                    ybit = __ffsll(Ac) - 1;
                    Ac &= Ac - 1;
                    y = (ybit >= 32 ? n : 0) + nc + (ybit & 31);
                }
                unsigned long long kact = AO;
                if (xbit >= 0) kact &= ~(1ull << xbit);
                if (ybit >= 0) kact |= (1ull << ybit);
                ctr.cand();
                const unsigned long long key = hash_key(S, (unsigned)kact, (unsigned)(kact >> 32));
                if (key == self_key) {
                    acc += self_term;
                    ctr.term();
                    continue;
                }
                double c = hash_lookup(S, key, ctr);
                if ((__double_as_longlong(c) << 1) != 0) {          // c != 0 without an FP64 compare
                    acc += (G.g ? single_from_walker<W>(S, G, m, x, y, ctr) : single_elem<W>(S, m, x, y, ctr)) * c;
                    ctr.term();
                }
            }
        }
    }
    // r = 2
    {
        const int ne = 2 - pc, nf = 2 - hc;   // extra active electrons removed / holes filled
        // enumerate extra removals (subsets of AO of size ne)
        unsigned long long r1set = (ne >= 1) ? AO : 1ull;
        while (r1set) {
            int b1 = -1;
            unsigned long long rest = 0;
            if (ne >= 1) {
                b1 = __ffsll(r1set) - 1;
                r1set &= r1set - 1;
                rest = r1set;           // second extra removal from bits above b1
            } else {
                r1set = 0;
            }
            unsigned long long r2set = (ne == 2) ? rest : 1ull;
            while (r2set) {
                int b2 = -1;
                if (ne == 2) {
                    b2 = __ffsll(r2set) - 1;
                    r2set &= r2set - 1;
                } else {
                    r2set = 0;
                }
                // removed spin orbitals and their alpha count
                int R[2], nr = 0, ra = pa;
                for (int i = 0; i < pc; i++) R[nr++] = ps[i];
                if (b1 >= 0) { R[nr++] = (b1 >= 32 ? n : 0) + nc + (b1 & 31); ra += b1 < 32; }
                if (b2 >= 0) { R[nr++] = (b2 >= 32 ? n : 0) + nc + (b2 & 31); ra += b2 < 32; }
                unsigned long long rbits = (b1 >= 0 ? (1ull << b1) : 0ull) | (b2 >= 0 ? (1ull << b2) : 0ull);
                // extra fillings: subsets of AE of size nf, alpha count must make ha + fa == ra
                unsigned long long a1set = (nf >= 1) ? AE : 1ull;
                while (a1set) {
                    int c1 = -1;
                    unsigned long long rest2 = 0;
                    if (nf >= 1) {
                        c1 = __ffsll(a1set) - 1;
                        a1set &= a1set - 1;
                        rest2 = a1set;
                    } else {
                        a1set = 0;
                    }
                    unsigned long long a2set = (nf == 2) ? rest2 : 1ull;
                    while (a2set) {
                        int c2 = -1;
                        if (nf == 2) {
                            c2 = __ffsll(a2set) - 1;
                            a2set &= a2set - 1;
                        } else {
                            a2set = 0;
                        }
                        int fa = ha + (c1 >= 0 && c1 < 32) + (c2 >= 0 && c2 < 32);
                        if (fa != ra) continue;
                        int A[2], nA = 0;
                        for (int i = 0; i < hc; i++) A[nA++] = hs[i];
                        if (c1 >= 0) A[nA++] = (c1 >= 32 ? n : 0) + nc + (c1 & 31);
                        if (c2 >= 0) A[nA++] = (c2 >= 32 ? n : 0) + nc + (c2 & 31);
                        unsigned long long abits = (c1 >= 0 ? (1ull << c1) : 0ull) | (c2 >= 0 ? (1ull << c2) : 0ull);
                        unsigned long long kact = (AO & ~rbits) | abits;
                        ctr.cand();
                        const unsigned long long key = hash_key(S, (unsigned)kact, (unsigned)(kact >> 32));
                        if (key == self_key) {
                            acc += self_term;
                            ctr.term();
                            continue;
                        }
                        double c = hash_lookup(S, key, ctr);
                        if ((__double_as_longlong(c) << 1) == 0) continue;
                        ctr.term();
                        int r1 = R[0] < R[1] ? R[0] : R[1], r2 = R[0] < R[1] ? R[1] : R[0];
                        int a1 = A[0] < A[1] ? A[0] : A[1], a2 = A[0] < A[1] ? A[1] : A[0];
                        acc += hb_screen(S, double_elem<W>(S, m, r1, r2, a1, a2, ctr)) * c;
                    }
                }
            }
        }
    }
    return acc;
}

// ------------------------------------------------------------------ Philox4x32-10

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        uint4 o;
        o.x = hi1 ^ c.y ^ k.x;
        o.y = lo1;
        o.z = hi0 ^ c.w ^ k.y;
        o.w = lo0;
        c = o;
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// 53 random bits k of Philox(seed; exc, step, walker, 0); the uniform is u = (k+1) 2^-53 in (0,1]
__device__ __forceinline__ unsigned long long race_bits(unsigned long long seed, unsigned exc, unsigned step,
                                                        unsigned walker) {
    uint4 o = philox4x32_10(make_uint4(exc, step, walker, 0u), make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
    return ((((unsigned long long)o.x) << 32) | o.y) >> 11;
}

// exponential clock of the first-reaction form of Gillespie's algorithm: t = -ln(u)/rate
__device__ __forceinline__ double race_clock_f64(unsigned long long k, double rate) {
    const double u = (double)(k + 1) * (1.0 / 9007199254740992.0);
    return -log(u) / rate;
}

// FP32 image of |x| from its bits (mantissa truncated to 23 bits, relative error < 2^-23); 0 outside
// [2^-100, 2^100]
__device__ __forceinline__ float abs_f32_of(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32) & 0x7FFFFFFFu;
    const int e = (int)(hi >> 20);                       // biased exponent
    if (e < 1023 - 100 || e > 1023 + 100) return 0.0f;
    const unsigned f = ((unsigned)(e - 1023 + 127) << 23) | ((hi & 0xFFFFFu) << 3) | (unsigned)((b & 0xFFFFFFFFull) >> 29);
    return __uint_as_float(f);
}

// The race's screen: can a neighbour with rate Gamma (FP32 image gf) and random bits k beat the best
// clock t_best so far (FP32 image btf)?  Its exact clock -ln(u)/Gamma wins iff u > exp(-Gamma t_best),
// i.e. iff w = 1 - u = (2^53 - 1 - k) 2^-53 < -expm1(-Gamma t_best).  With y = gf btf (1 + 1e-4),
// which exceeds Gamma t_best despite the FP32 roundings, and y <= 4, the test w < -expm1(-y) has
// a relative margin above 1.8e-6, far above the FP32 errors (about 2e-7), so it never rejects a
// winner; for y > 4, for gf, btf or y outside the normal FP32 range and with no best yet it lets every
// candidate through, and the exact FP64 clock decides.  No logarithm and no division per neighbour.
__device__ __forceinline__ bool race_may_win(unsigned long long k, float gf, float btf) {
    if (!(gf >= 1e-30f) || !(btf >= 1e-30f)) return true;
    const float y = gf * btf * 1.0001f;
    if (!(y >= 1e-30f && y <= 4.0f)) return true;
    return (float)(9007199254740991ull - k) * 1.1102230246251565e-16f < -expm1f(-y);
}
