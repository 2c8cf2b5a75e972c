// mrq.cu - GB300 (sm_103a) kernels and host runtime of the stochastic SC-NEVPT2(s) /
// SC-MRCI(s) local-estimator path (arXiv:1909.06935), behind the C ABI of include/mrq.h.
//
// Hot path (one warp per walker, persistent over steps):
//   classify the walker (label, Sec. II A) -> enumerate every single and double excitation that
//   stays in CAS u FOIS as a union of rectangular class blocks -> per lane: <n|H|m> by
//   Slater-Condon, psi_s(m) by a hash probe (m in the CAS) or reach-back O(m) = <m|H|phi0>
//   (Eq. 6-7, Sec. II D) -> rates Gamma_nm = |H_nm psi_s(m)/psi_s(n)|, E_L (Eq. 5), the H_D
//   numerator (Eq. 16) -> warp reductions -> accumulate with weight 1/S -> move by the
//   first-reaction (competing exponential clocks) form of Gillespie's algorithm.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <chrono>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/mrq.h"
#include "mrq_device.cuh"
#include "mrq_internal.h"

// ============================================================================ per-warp state

struct Walker {
    unsigned long long d[2][2];   // [spin][word]
    double psi;                   // psi_s of the current determinant
    unsigned step;                // steps taken by this walker so far
    unsigned wid;                 // walker id (Philox counter word)
    int sys;                      // index into the system table
    int group;                    // accumulator group
    // the last step's contribution, written by the walk and added by k_accum
    long long rl;                 // label of the determinant the step was taken at (-1: nothing to add)
    double rw, rEL, rnum;         // residence weight 1/S, E_L, H_D numerator
    int rtype;                    // 3h + p
    int rpad;
};

static_assert(sizeof(SysDev) % sizeof(int) == 0, "SysDev is copied word by word");

struct WarpSh {
    SysDev sys;                      // the walker's system, read by every lane (kept out of local memory)
    unsigned char ol[2][MRQ_MAXN];   // occupied orbitals per spin, ascending (core|active|virtual)
    unsigned char el[2][MRQ_MAXN];   // empty orbitals per spin
    short os[2][4], es[2][4];        // class starts: [spin][class], [3] = count
    int bstart[MRQ_MAXB + 1];        // block prefix offsets
    unsigned bdesc[MRQ_MAXB];        // block descriptors
    int nb;
};

// pair tables for same-spin doubles: (X1, X2) with X1 <= X2
__constant__ unsigned char c_pair_a[6] = {0, 0, 0, 1, 1, 2};
__constant__ unsigned char c_pair_b[6] = {0, 1, 2, 1, 2, 2};

__device__ __forceinline__ int pairs_of(int k1, int k2, bool same) { return same ? k1 * (k1 - 1) / 2 : k1 * k2; }

// enumeration speed of an orbital class: active slowest (0), core (1), virtual fastest (2)
__device__ __forceinline__ int cls_pri(int c) { return c == 1 ? 0 : (c == 0 ? 1 : 2); }

// pair index -> (i < j), ordered by j then i (used for the occupied-pair diagonal sums)
__device__ __forceinline__ void tri_decode(int op, int& i, int& j) {
    int jj = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)op)) * 0.5f);
    while (jj * (jj - 1) / 2 > op) jj--;
    while ((jj + 1) * jj / 2 <= op) jj++;
    j = jj;
    i = op - jj * (jj - 1) / 2;
}

// Build occupied/empty lists (class-partitioned) and the valid excitation blocks of det d.
template <int W>
__device__ void build_lists(const SysDev& S, const unsigned long long (&d)[2][W], WarpSh& sh, int h, int p,
                            int lane) {
    const int n = S.n;
    for (int sg = 0; sg < 2; sg++) {
        int no = 0, ne = 0;
        for (int base = 0; base < n; base += 32) {
            int q = base + lane;
            bool valid = q < n;
            bool o = valid && bit_of<W>(d[sg], q);
            unsigned bo = __ballot_sync(0xffffffffu, o);
            unsigned be = __ballot_sync(0xffffffffu, valid && !o);
            unsigned lt = (1u << lane) - 1u;
            if (o) sh.ol[sg][no + __popc(bo & lt)] = (unsigned char)q;
            if (valid && !o) sh.el[sg][ne + __popc(be & lt)] = (unsigned char)q;
            no += __popc(bo);
            ne += __popc(be);
        }
        if (lane == 0) {
            int oc = 0, oa = 0, ov = 0;
#pragma unroll
            for (int w = 0; w < W; w++) {
                oc += __popcll(d[sg][w] & S.mcore[w]);
                oa += __popcll(d[sg][w] & S.mact[w]);
                ov += __popcll(d[sg][w] & S.mvirt[w]);
            }
            sh.os[sg][0] = 0;
            sh.os[sg][1] = oc;
            sh.os[sg][2] = oc + oa;
            sh.os[sg][3] = oc + oa + ov;
            sh.es[sg][0] = 0;
            sh.es[sg][1] = S.nc - oc;
            sh.es[sg][2] = S.nc - oc + S.na - oa;
            sh.es[sg][3] = n - (oc + oa + ov);
        }
    }
    __syncwarp();
    // candidate blocks: 18 singles, 72 same-spin doubles, 81 opposite-spin doubles
    int run = 0, carry = 0;
    for (int base = 0; base < MRQ_MAXB; base += 32) {
        int ci = base + lane;
        int size = 0, kind = 0, sg = 0, X1 = 0, X2 = 0, Y1 = 0, Y2 = 0;
        unsigned order = 0;
        if (ci < MRQ_MAXB) {
            if (ci < 18) {
                kind = 0; sg = ci / 9; X1 = (ci % 9) / 3; Y1 = ci % 3;
                size = (sh.os[sg][X1 + 1] - sh.os[sg][X1]) * (sh.es[sg][Y1 + 1] - sh.es[sg][Y1]);
            } else if (ci < 90) {
                int c = ci - 18;
                kind = 1; sg = c / 36;
                int px = (c % 36) / 6, py = c % 6;
                X1 = c_pair_a[px]; X2 = c_pair_b[px]; Y1 = c_pair_a[py]; Y2 = c_pair_b[py];
                int k1 = sh.os[sg][X1 + 1] - sh.os[sg][X1], k2 = sh.os[sg][X2 + 1] - sh.os[sg][X2];
                int e1 = sh.es[sg][Y1 + 1] - sh.es[sg][Y1], e2 = sh.es[sg][Y2 + 1] - sh.es[sg][Y2];
                size = pairs_of(k1, k2, X1 == X2) * pairs_of(e1, e2, Y1 == Y2);
            } else {
                int c = ci - 90;
                kind = 2; X1 = c / 27; Y1 = (c / 9) % 3; X2 = (c / 3) % 3; Y2 = c % 3;
                size = (sh.os[0][X1 + 1] - sh.os[0][X1]) * (sh.es[0][Y1 + 1] - sh.es[0][Y1]) *
                       (sh.os[1][X2 + 1] - sh.os[1][X2]) * (sh.es[1][Y2 + 1] - sh.es[1][Y2]);
            }
            // digit order inside the block: active indices slowest, core next, virtual fastest, so
            // that the lanes of one warp iteration share the active remnant of their neighbours
            if (kind == 0) {
                order = cls_pri(X1) > cls_pri(Y1) ? 1u : 0u;                         // occ fastest?
            } else if (kind == 1) {
                int po = min(cls_pri(X1), cls_pri(X2)), pe = min(cls_pri(Y1), cls_pri(Y2));
                order = (pe < po ? 1u : 0u) | ((X1 != X2 && cls_pri(X1) > cls_pri(X2)) ? 2u : 0u) |
                        ((Y1 != Y2 && cls_pri(Y1) > cls_pri(Y2)) ? 4u : 0u);
            } else {
                int cl[4] = {X1, Y1, X2, Y2}, perm[4] = {0, 1, 2, 3};
                for (int a = 1; a < 4; a++)       // stable insertion sort by class priority
                    for (int b2 = a; b2 > 0 && cls_pri(cl[perm[b2]]) < cls_pri(cl[perm[b2 - 1]]); b2--) {
                        int t = perm[b2]; perm[b2] = perm[b2 - 1]; perm[b2 - 1] = t;
                    }
                order = (unsigned)perm[0] | ((unsigned)perm[1] << 2) | ((unsigned)perm[2] << 4) |
                        ((unsigned)perm[3] << 6);
            }
            int dh = (X1 == 0) - (Y1 == 0), dp = (Y1 == 2) - (X1 == 2);
            if (kind != 0) {
                dh += (X2 == 0) - (Y2 == 0);
                dp += (Y2 == 2) - (X2 == 2);
            }
            if (h + dh > 2 || p + dp > 2) size = 0;
        }
        unsigned vm = __ballot_sync(0xffffffffu, size > 0);
        // inclusive scan of sizes (invalid lanes contribute 0) -> global prefix via the carry
        int x = size;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (size > 0) {
            int k = run + __popc(vm & ((1u << lane) - 1u));
            sh.bdesc[k] = (unsigned)kind | ((unsigned)sg << 2) | ((unsigned)X1 << 4) | ((unsigned)X2 << 6) |
                          ((unsigned)Y1 << 8) | ((unsigned)Y2 << 10) | (order << 12);
            sh.bstart[k + 1] = carry + x;
        }
        carry += __shfl_sync(0xffffffffu, x, 31);
        run += __popc(vm);
    }
    if (lane == 0) {
        sh.nb = run;
        sh.bstart[0] = 0;
    }
    __syncwarp();
}

// pair index -> (i < j) in lexicographic order (i slowest, j fastest) among k items
__device__ __forceinline__ void lex_decode(int op, int k, int& i, int& j) {
    int ti, tj;
    tri_decode(k * (k - 1) / 2 - 1 - op, ti, tj);
    i = k - 1 - tj;
    j = k - 1 - ti;
}

// pair within one class (lexicographic) or across two classes (rev: first index fastest)
__device__ __forceinline__ void pair_decode(int op, bool same, int k1, int k2, bool rev, int& i, int& j) {
    if (same) lex_decode(op, k1, i, j);
    else if (rev) { j = op / k1; i = op - j * k1; }
    else { i = op / k2; j = op - i * k2; }
}

// decode neighbour `loc` of block `desc` into removed r1<=r2 and added a1<=a2 spin orbitals
__device__ __forceinline__ void decode_exc(const WarpSh& sh, int n, unsigned desc, int loc, int& kind, int& r1,
                                           int& r2, int& a1, int& a2) {
    kind = desc & 3;
    int sg = (desc >> 2) & 1, X1 = (desc >> 4) & 3, X2 = (desc >> 6) & 3, Y1 = (desc >> 8) & 3,
        Y2 = (desc >> 10) & 3;
    const unsigned order = desc >> 12;
    if (kind == 0) {
        int nX = sh.os[sg][X1 + 1] - sh.os[sg][X1], nY = sh.es[sg][Y1 + 1] - sh.es[sg][Y1];
        int i, a;
        if (order & 1u) { a = loc / nX; i = loc - a * nX; }
        else { i = loc / nY; a = loc - i * nY; }
        r1 = r2 = sg * n + sh.ol[sg][sh.os[sg][X1] + i];
        a1 = a2 = sg * n + sh.el[sg][sh.es[sg][Y1] + a];
    } else if (kind == 1) {
        int k1 = sh.os[sg][X1 + 1] - sh.os[sg][X1], k2 = sh.os[sg][X2 + 1] - sh.os[sg][X2];
        int e1 = sh.es[sg][Y1 + 1] - sh.es[sg][Y1], e2 = sh.es[sg][Y2 + 1] - sh.es[sg][Y2];
        int nOP = pairs_of(k1, k2, X1 == X2), nEP = pairs_of(e1, e2, Y1 == Y2);
        int op, ep;
        if (order & 1u) { ep = loc / nOP; op = loc - ep * nOP; }
        else { op = loc / nEP; ep = loc - op * nEP; }
        int i, j, a, b;
        pair_decode(op, X1 == X2, k1, k2, (order & 2u) != 0, i, j);
        pair_decode(ep, Y1 == Y2, e1, e2, (order & 4u) != 0, a, b);
        r1 = sg * n + sh.ol[sg][sh.os[sg][X1] + i];
        r2 = sg * n + sh.ol[sg][sh.os[sg][X2] + j];
        a1 = sg * n + sh.el[sg][sh.es[sg][Y1] + a];
        a2 = sg * n + sh.el[sg][sh.es[sg][Y2] + b];
    } else {
        // digits 0: alpha occupied (X1), 1: alpha empty (Y1), 2: beta occupied (X2), 3: beta empty (Y2)
        int rad[4] = {sh.os[0][X1 + 1] - sh.os[0][X1], sh.es[0][Y1 + 1] - sh.es[0][Y1],
                      sh.os[1][X2 + 1] - sh.os[1][X2], sh.es[1][Y2 + 1] - sh.es[1][Y2]};
        int x[4];
#pragma unroll
        for (int d = 3; d >= 0; d--) {
            int id = (order >> (2 * d)) & 3u;
            int q = loc / rad[id];
            x[id] = loc - q * rad[id];
            loc = q;
        }
        r1 = sh.ol[0][sh.os[0][X1] + x[0]];
        a1 = sh.el[0][sh.es[0][Y1] + x[1]];
        r2 = n + sh.ol[1][sh.os[1][X2] + x[2]];
        a2 = n + sh.el[1][sh.es[1][Y2] + x[3]];
    }
}

__device__ __forceinline__ bool active_only(unsigned desc) {
    int kind = desc & 3, X1 = (desc >> 4) & 3, X2 = (desc >> 6) & 3, Y1 = (desc >> 8) & 3, Y2 = (desc >> 10) & 3;
    if (kind == 0) return X1 == 1 && Y1 == 1;
    return X1 == 1 && X2 == 1 && Y1 == 1 && Y2 == 1;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// <d|H|d> and <d|H_D|d> (lane-parallel over occupied pairs); label >= 0 required for H_D
template <int W>
__device__ void diagonals(const SysDev& S, const WarpSh& sh, const unsigned long long (&d)[2][W], int lane,
                          double& hnn, double& hdnn) {
    const int na_ = sh.os[0][3], nb_ = sh.os[1][3], N = na_ + nb_;
    double h = 0.0, hd = 0.0;
    for (int k = lane; k < N; k += 32) {
        int p = k < na_ ? sh.ol[0][k] : sh.ol[1][k - na_];
        h += __ldg(S.h1 + p * S.n + p);
        int cls = p < S.nc ? 0 : (p < S.nc + S.na ? 1 : 2);
        if (cls == 1) hd += __ldg(S.hc + p * S.n + p);
        else if (cls == 2) hd += __ldg(S.eps + p);
    }
    // core holes
    for (int sg = 0; sg < 2; sg++) {
        for (int k = lane; k < S.nc - sh.os[sg][1]; k += 32) hd -= __ldg(S.eps + sh.el[sg][k]);
    }
    const int npair = N * (N - 1) / 2;
    for (int q = lane; q < npair; q += 32) {
        int j, i;
        tri_decode(q, i, j);
        int si = i >= na_, sj = j >= na_;
        int p1 = si ? sh.ol[1][i - na_] : sh.ol[0][i];
        int p2 = sj ? sh.ol[1][j - na_] : sh.ol[0][j];
        double v = eri_g(S, p1, p1, p2, p2);
        if (si == sj) v -= eri_g(S, p1, p2, p2, p1);
        h += v;
        bool a1 = p1 >= S.nc && p1 < S.nc + S.na, a2 = p2 >= S.nc && p2 < S.nc + S.na;
        if (a1 && a2) hd += v;
    }
    hnn = warp_sum(h) + S.e_nuc;
    hdnn = warp_sum(hd) + S.e_core;
}

// ============================================================================ the walk

enum { MODE_STEP = 0, MODE_DEBUG = 1 };

#include "mrq_cas.cuh"

// The walkers of one launch: one or several systems, each with its own walker array; slot numbers
// run over all systems (system k owns slots [offsets[k], offsets[k+1])).
struct WalkSet {
    const SysDev* systems;
    Walker* const* walkers;
    const long long* offsets;
    int nsys;
    long long nslots;
    long long max_seg = 0;        // the most slots of one system (host side: sizes the slot sort)
};

__device__ __forceinline__ void slot_owner(const WalkSet& ws, long long slot, int& sys, long long& local) {
    int lo = 0, hi = ws.nsys - 1;
    while (lo < hi) {                       // last system whose first slot is <= slot
        const int mid = (lo + hi + 1) >> 1;
        if (ws.offsets[mid] <= slot) lo = mid;
        else hi = mid - 1;
    }
    sys = lo;
    local = slot - ws.offsets[lo];
}

// sort key of a walker slot: system, label, then the active occupation (truncated), and the slot
template <int W>
__global__ void k_walker_keys(const WalkSet ws, unsigned long long* __restrict__ keys) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ws.nslots) return;
    int sys;
    long long local;
    slot_owner(ws, i, sys, local);
    const Walker wk = ws.walkers[sys][local];
    const SysDev& S = ws.systems[sys];
    unsigned long long d[2][W];
#pragma unroll
    for (int sg = 0; sg < 2; sg++)
#pragma unroll
        for (int w = 0; w < W; w++) d[sg][w] = wk.d[sg][w];
    int h, p;
    const long long l = det_label<W>(S, d, h, p);
    const unsigned long long act = hash_key(S, active_bits<W>(S, d[0]), active_bits<W>(S, d[1]));
    keys[i] = ((unsigned long long)(l & 0xFFFFFF) << 24) | (act & 0xFFFFFFull);
}

// Per-system bitonic sort of the slots by key (ties by slot): block b orders the slots of system b,
// [offsets[b], offsets[b+1]), in shared memory padded to a power of two; a system with fewer than
// 64 or more than MRQ_SORT_MAX slots keeps its slot order.  order[] receives global slot numbers.
#define MRQ_SORT_MAX 16384
__global__ void __launch_bounds__(1024) k_sort_slots(const unsigned long long* __restrict__ keys,
                                                     const long long* __restrict__ offsets, unsigned* __restrict__ order) {
    extern __shared__ __align__(16) unsigned char sort_smem[];
    const long long lo = offsets[blockIdx.x];
    const int n = (int)(offsets[blockIdx.x + 1] - lo);
    if (n < 64 || n > MRQ_SORT_MAX) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) order[lo + i] = (unsigned)(lo + i);
        return;
    }
    const int npad = 1 << (32 - __clz(n - 1));
    unsigned long long* sk = reinterpret_cast<unsigned long long*>(sort_smem);
    unsigned* si = reinterpret_cast<unsigned*>(sk + npad);
    for (int i = threadIdx.x; i < npad; i += blockDim.x) {
        sk[i] = i < n ? keys[lo + i] : ~0ull;
        si[i] = i < n ? (unsigned)(lo + i) : 0xFFFFFFFFu;
    }
    __syncthreads();
    for (int k = 2; k <= npad; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < npad; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const unsigned long long a = sk[i], b = sk[ixj];
                    const bool swap = up ? (a > b || (a == b && si[i] > si[ixj])) : (a < b || (a == b && si[i] < si[ixj]));
                    if (swap) {
                        sk[i] = b;
                        sk[ixj] = a;
                        const unsigned t = si[i];
                        si[i] = si[ixj];
                        si[ixj] = t;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) order[lo + i] = si[i];
}

#include "mrq_walk.cuh"

__global__ void k_walkers_init(Walker* w, long long nslots, unsigned long long d0, unsigned long long d1,
                               unsigned long long d2, unsigned long long d3, double psi, int sys, int G) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nslots) return;
    Walker x;
    x.d[0][0] = d0; x.d[0][1] = d1; x.d[1][0] = d2; x.d[1][1] = d3;
    x.psi = psi;
    x.step = 0;
    x.wid = (unsigned)i;
    x.sys = sys;
    x.group = (int)(i % G);
    x.rl = -1;
    x.rw = x.rEL = x.rnum = 0.0;
    x.rtype = 0;
    x.rpad = 0;
    w[i] = x;
}

// ============================================================================ setup kernels

// insert reference determinants (and validate them: full core, empty virtuals, electron counts)
template <int W>
__global__ void k_hash_build(const SysDev* __restrict__ sys, HashSlot* __restrict__ hash, const unsigned long long* dets,
                             const double* coeffs, long long nref, int* err) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nref) return;
    const SysDev S = *sys;
    unsigned long long d[2][W];
#pragma unroll
    for (int w = 0; w < W; w++) {
        d[0][w] = dets[i * 2 * W + w];
        d[1][w] = dets[i * 2 * W + W + w];
    }
    int ca = 0, cb = 0;
    bool bad = false;
#pragma unroll
    for (int w = 0; w < W; w++) {
        ca += __popcll(d[0][w]);
        cb += __popcll(d[1][w]);
        unsigned long long all = S.mcore[w] | S.mact[w] | S.mvirt[w];
        for (int sg = 0; sg < 2; sg++) {
            if ((d[sg][w] & S.mcore[w]) != S.mcore[w]) bad = true;
            if (d[sg][w] & S.mvirt[w]) bad = true;
            if (d[sg][w] & ~all) bad = true;
        }
    }
    if (ca != S.nalpha || cb != S.nbeta) bad = true;
    if (bad) {
        atomicOr(err, 8);
        return;
    }
    unsigned long long key = hash_key(S, active_bits<W>(S, d[0]), active_bits<W>(S, d[1]));
    unsigned long long hidx = mix64(key) & S.hmask;
    for (int k = 0; k < S.max_probe; k++) {
        unsigned long long prev = atomicCAS(&hash[hidx].key, MRQ_EMPTY_KEY, key);
        if (prev == MRQ_EMPTY_KEY) {
            hash[hidx].val = coeffs[i];
            return;
        }
        if (prev == key) {
            atomicOr(err, 16);   // duplicate determinant
            return;
        }
        hidx = (hidx + 1) & S.hmask;
    }
    atomicOr(err, 32);   // probe bound exceeded
}

__global__ void k_hash_clear(HashSlot* hash, unsigned long long cap) {
    unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cap) {
        hash[i].key = MRQ_EMPTY_KEY;
        hash[i].val = 0.0;
    }
}

// half-unpacked integral table E[P(p,q)][r][s] from the 8-fold packed input
__global__ void k_expand_eri(const double* __restrict__ eri, double* __restrict__ eri4, int n) {
    const long long npair = (long long)n * (n + 1) / 2;
    const long long total = npair * n * n;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        long long P = t / ((long long)n * n);
        int rs = (int)(t - P * n * n);
        int r = rs / n, s = rs - r * n;
        long long Q = r >= s ? (long long)r * (r + 1) / 2 + s : (long long)s * (s + 1) / 2 + r;
        long long i = P >= Q ? P * (P + 1) / 2 + Q : Q * (Q + 1) / 2 + P;
        eri4[t] = eri[i];
    }
}

// physicists' tables on the (core+active) x (core+active) x (active+virtual) x (active+virtual)
// block: T[p][q][r][s] = <pq|rs> = (pr|qs) and, after tab_half entries, <pq||rs>
__global__ void k_build_tab(const SysDev* __restrict__ sys, double* __restrict__ tab) {
    const SysDev S = *sys;
    const long long a = S.nca, v = S.nav, half = a * a * v * v;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < half; t += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(t % v) + S.nc, r = (int)((t / v) % v) + S.nc;
        const int q = (int)((t / (v * v)) % a), p = (int)(t / (v * v * a));
        const double d = eri_g(S, p, r, q, s), x = eri_g(S, p, s, q, r);
        tab[t] = hb_screen(S, d);                 // every double the CAS path takes reads one entry
        tab[half + t] = hb_screen(S, d - x);
    }
}

// hc_pq = h_pq + sum_i [2(pq|ii) - (pi|iq)]
__global__ void k_core_fock(const SysDev* __restrict__ sys, double* hc) {
    const SysDev S = *sys;
    int pq = blockIdx.x * blockDim.x + threadIdx.x;
    if (pq >= S.n * S.n) return;
    int p = pq / S.n, q = pq % S.n;
    double v = __ldg(S.h1 + pq);
    for (int i = 0; i < S.nc; i++) v += 2.0 * eri_g(S, p, q, i, i) - eri_g(S, p, i, i, q);
    hc[pq] = v;
}

// block-level deterministic sum of `nv` values per thread into out[blockIdx.x * nv + k]
template <int NV>
__device__ void block_sum_store(double (&v)[NV], double* out) {
    __shared__ double red[32][NV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double x = warp_sum(v[k]);
        if (lane == 0) red[wid][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < nw; w++) s += red[w][threadIdx.x];
        out[(long long)blockIdx.x * NV + threadIdx.x] = s;
    }
    __syncthreads();
}

// E0 numerator and norm: sum_k c_k^2 H_kk + sum_k sum_{k' active exc} c_k H_kk' c_k'
// one thread per (reference determinant, excitation) pair, strided; partials per block.
template <int W>
__global__ void k_ref_energy(const SysDev* __restrict__ sys, const unsigned long long* dets, const double* coeffs,
                             long long nref, double* partial) {
    const SysDev S = *sys;
    double acc[2] = {0.0, 0.0};
    const int na = S.na;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gsz = (long long)gridDim.x * blockDim.x;
    for (long long i = gtid; i < nref; i += gsz) {
        unsigned long long d[2][W];
#pragma unroll
        for (int w = 0; w < W; w++) {
            d[0][w] = dets[i * 2 * W + w];
            d[1][w] = dets[i * 2 * W + W + w];
        }
        const double ck = coeffs[i];
        acc[1] += ck * ck;
        // diagonal
        double hdiag = S.e_nuc;
        for (int sg = 0; sg < 2; sg++)
            for (int w = 0; w < W; w++) {
                unsigned long long om = d[sg][w];
                while (om) {
                    int p1 = 64 * w + __ffsll(om) - 1;
                    om &= om - 1;
                    hdiag += __ldg(S.h1 + p1 * S.n + p1);
                    for (int sg2 = 0; sg2 < 2; sg2++)
                        for (int w2 = 0; w2 < W; w2++) {
                            unsigned long long om2 = d[sg2][w2];
                            while (om2) {
                                int p2 = 64 * w2 + __ffsll(om2) - 1;
                                om2 &= om2 - 1;
                                hdiag += 0.5 * eri_g(S, p1, p1, p2, p2);
                                if (sg == sg2) hdiag -= 0.5 * eri_g(S, p1, p2, p2, p1);
                            }
                        }
                }
            }
        double off = 0.0;
        const unsigned ao[2] = {active_bits<W>(S, d[0]), active_bits<W>(S, d[1])};
        const unsigned am = (na >= 32) ? 0xFFFFFFFFu : ((1u << na) - 1u);
        // singles and same-spin doubles
        for (int sg = 0; sg < 2; sg++) {
            unsigned o1 = ao[sg];
            while (o1) {
                int t = __ffs(o1) - 1;
                o1 &= o1 - 1;
                unsigned e1 = ~ao[sg] & am;
                while (e1) {
                    int u = __ffs(e1) - 1;
                    e1 &= e1 - 1;
                    unsigned k0 = ao[0], k1 = ao[1];
                    (sg ? k1 : k0) ^= (1u << t) | (1u << u);
                    double c = hash_lookup(S, hash_key(S, k0, k1));
                    NoCtr z;
                    if (c != 0.0) off += ck * c * single_elem<W>(S, d, sg * S.n + S.nc + t, sg * S.n + S.nc + u, z);
                }
                unsigned o2 = o1;   // t2 > t
                while (o2) {
                    int t2 = __ffs(o2) - 1;
                    o2 &= o2 - 1;
                    unsigned e2 = ~ao[sg] & am;
                    while (e2) {
                        int u1 = __ffs(e2) - 1;
                        e2 &= e2 - 1;
                        unsigned e3 = e2;
                        while (e3) {
                            int u2 = __ffs(e3) - 1;
                            e3 &= e3 - 1;
                            unsigned k0 = ao[0], k1 = ao[1];
                            (sg ? k1 : k0) ^= (1u << t) | (1u << t2) | (1u << u1) | (1u << u2);
                            double c = hash_lookup(S, hash_key(S, k0, k1));
                            if (c != 0.0) {
                                int b = sg * S.n + S.nc;
                                NoCtr z;
                                off += ck * c * double_elem<W>(S, d, b + t, b + t2, b + u1, b + u2, z);
                            }
                        }
                    }
                }
            }
        }
        // opposite-spin doubles
        {
            unsigned oa = ao[0];
            while (oa) {
                int t = __ffs(oa) - 1;
                oa &= oa - 1;
                unsigned ea = ~ao[0] & am;
                while (ea) {
                    int u = __ffs(ea) - 1;
                    ea &= ea - 1;
                    unsigned ob = ao[1];
                    while (ob) {
                        int s = __ffs(ob) - 1;
                        ob &= ob - 1;
                        unsigned eb = ~ao[1] & am;
                        while (eb) {
                            int v = __ffs(eb) - 1;
                            eb &= eb - 1;
                            unsigned k0 = ao[0] ^ ((1u << t) | (1u << u));
                            unsigned k1 = ao[1] ^ ((1u << s) | (1u << v));
                            double c = hash_lookup(S, hash_key(S, k0, k1));
                            NoCtr z;
                            if (c != 0.0)
                                off += ck * c *
                                       double_elem<W>(S, d, S.nc + t, S.n + S.nc + s, S.nc + u, S.n + S.nc + v, z);
                        }
                    }
                }
            }
        }
        acc[0] += ck * ck * hdiag + off;
    }
    block_sum_store<2>(acc, partial);
}

// spin-summed active 1-RDM element gamma_tu (unnormalised): block (t, u) over all determinants
template <int W>
__global__ void k_ref_rdm(const SysDev* __restrict__ sys, const unsigned long long* dets, const double* coeffs,
                          long long nref, double* gamma_raw) {
    const SysDev S = *sys;
    const int t = blockIdx.x / S.na, u = blockIdx.x % S.na;
    double acc[1] = {0.0};
    for (long long i = threadIdx.x; i < nref; i += blockDim.x) {
        unsigned long long d[2][W];
#pragma unroll
        for (int w = 0; w < W; w++) {
            d[0][w] = dets[i * 2 * W + w];
            d[1][w] = dets[i * 2 * W + W + w];
        }
        const double ck = coeffs[i];
        const unsigned ao[2] = {active_bits<W>(S, d[0]), active_bits<W>(S, d[1])};
        for (int sg = 0; sg < 2; sg++) {
            // <phi0| a+_t a_u |phi0>: d has u occupied; k' = d - u + t
            if (!((ao[sg] >> u) & 1u)) continue;
            if (t == u) {
                acc[0] += ck * ck;
                continue;
            }
            if ((ao[sg] >> t) & 1u) continue;
            unsigned k0 = ao[0], k1 = ao[1];
            (sg ? k1 : k0) ^= (1u << t) | (1u << u);
            double c = hash_lookup(S, hash_key(S, k0, k1));
            if (c != 0.0) acc[0] += ck * c * sgn_single<W>(d[sg], S.nc + u, S.nc + t);
        }
    }
    // single block per (t,u): reduce and store
    __shared__ double red[32];
    double x = warp_sum(acc[0]);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; w++) s += red[w];
        gamma_raw[blockIdx.x] = s;
    }
}

// reduce E0 partials (fixed order), normalise gamma, eps_p = F_pp, E_core; writes scal[0..4]
__global__ void k_setup_finish(const SysDev* __restrict__ sys, const double* partial, int npart, double* gamma,
                               double* eps, double* scal) {
    const SysDev S = *sys;
    __shared__ double s_num, s_norm;
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < npart; i++) {
            a += partial[2 * i];
            b += partial[2 * i + 1];
        }
        s_num = a;
        s_norm = b;
    }
    __syncthreads();
    const int na = S.na;
    for (int k = threadIdx.x; k < na * na; k += blockDim.x) gamma[k] /= s_norm;
    __syncthreads();
    for (int p = threadIdx.x; p < S.n; p += blockDim.x) {
        double v = __ldg(S.hc + p * S.n + p);
        for (int t = 0; t < na; t++)
            for (int u = 0; u < na; u++)
                v += gamma[t * na + u] * (eri_g(S, p, p, S.nc + t, S.nc + u) - 0.5 * eri_g(S, p, S.nc + t, S.nc + u, p));
        eps[p] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ec = S.e_nuc, se = 0.0;
        for (int i = 0; i < S.nc; i++) {
            ec += 2.0 * __ldg(S.h1 + i * S.n + i);
            for (int j = 0; j < S.nc; j++) ec += 2.0 * eri_g(S, i, i, j, j) - eri_g(S, i, j, j, i);
            se += eps[i];
        }
        scal[0] = s_num / s_norm;
        scal[1] = s_norm;
        scal[2] = ec;
        scal[3] = se;
    }
}

// the race's screen and exact clock for given (k, rate, best clock) triples (parity of the move
// selection's screen); the screen takes the FP32 images exactly as the walk forms them
__global__ void k_race_screen(const unsigned long long* __restrict__ k, const double* __restrict__ rate,
                              const double* __restrict__ tbest, long long n, unsigned char* __restrict__ pass,
                              double* __restrict__ exact) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float btf = isinf(tbest[i]) ? INFINITY : (float)tbest[i];
    pass[i] = race_may_win(k[i], abs_f32_of(rate[i]), btf) ? 1 : 0;
    exact[i] = race_clock_f64(k[i], rate[i]);
}

// index of the largest |c| (first on ties), one block
__global__ void k_argmax_abs(const double* c, long long n, long long* out) {
    __shared__ double bv[1024];
    __shared__ long long bi[1024];
    double v = -1.0;
    long long idx = 0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        double a = fabs(c[i]);
        if (a > v) { v = a; idx = i; }
    }
    bv[threadIdx.x] = v;
    bi[threadIdx.x] = idx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            double v2 = bv[threadIdx.x + s];
            long long i2 = bi[threadIdx.x + s];
            if (v2 > bv[threadIdx.x] || (v2 == bv[threadIdx.x] && i2 < bi[threadIdx.x])) {
                bv[threadIdx.x] = v2;
                bi[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = bi[0];
}

// ============================================================================ finalize (Eq. 14-15)

#define FIN_Q 5    // per type: kept ratio, e2, screened count, screened ratio, visited count
#define FIN_NV (MRQ_NTYPES * FIN_Q)

__device__ __forceinline__ int label_type(long long l, long long nPs, int nc2, int nv2) {
    long long rh = l / nPs, rp = l - rh * nPs;
    int h = rh == 0 ? 0 : (rh <= nc2 ? 1 : 2);
    int p = rp == 0 ? 0 : (rp <= nv2 ? 1 : 2);
    return 3 * h + p;
}

// block (v, chunk): labels of the chunk under variant v (v < G: group v left out; v == G: all)
__global__ void __launch_bounds__(256) k_fin_labels(const SysDev* __restrict__ sys, double tau, int nchunk,
                                                    long long chunk, double* partial) {
    const SysDev S = *sys;
    const int v = blockIdx.x / nchunk, ch = blockIdx.x % nchunk;
    const int G = S.G;
    const long long L = S.nlab;
    __shared__ double s_n0;
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int g = 0; g < G; g++) a += S.accN[(long long)g * L];
        if (v < G) a -= S.accN[(long long)v * L];
        s_n0 = a;
    }
    __syncthreads();
    const double n0 = s_n0;
    double acc[FIN_NV];
#pragma unroll
    for (int k = 0; k < FIN_NV; k++) acc[k] = 0.0;
    const long long lo = (long long)ch * chunk, hi = min(L, lo + chunk);
    for (long long l = lo + threadIdx.x; l < hi; l += blockDim.x) {
        if (l == 0) continue;
        double Nl = 0.0, Ul = 0.0;
        for (int g = 0; g < G; g++) {
            Nl += S.accN[(long long)g * L + l];
            Ul += S.accU[(long long)g * L + l];
        }
        if (v < G) {
            Nl -= S.accN[(long long)v * L + l];
            Ul -= S.accU[(long long)v * L + l];
        }
        if (!(Nl > 0.0)) continue;
        const int t = label_type(l, S.nPs, 2 * S.nc, 2 * S.nv);
        const double ratio = Nl / n0;
        double q[FIN_Q] = {0.0, 0.0, 0.0, 0.0, 1.0};
        if (ratio >= tau) {
            const double El = Ul / Nl;
            q[0] = ratio;
            q[1] = ratio / (S.e0 - El);
        } else {
            q[2] = 1.0;
            q[3] = ratio;
        }
#pragma unroll
        for (int tt = 0; tt < MRQ_NTYPES; tt++)
            if (tt == t) {
#pragma unroll
                for (int k = 0; k < FIN_Q; k++) acc[tt * FIN_Q + k] += q[k];
            }
    }
    block_sum_store<FIN_NV>(acc, partial);
}

// one block: sum chunk partials in order, jackknife over groups, write the result struct
__global__ void k_fin_reduce(const SysDev* __restrict__ sys, const double* partial, int nchunk, mrq_result* res) {
    const SysDev S = *sys;
    const int G = S.G;
    const long long L = S.nlab;
    __shared__ double vals[65][FIN_NV];   // G <= 64
    for (int idx = threadIdx.x; idx < (G + 1) * FIN_NV; idx += blockDim.x) {
        int v = idx / FIN_NV, k = idx % FIN_NV;
        double s = 0.0;
        for (int c = 0; c < nchunk; c++) s += partial[((long long)v * nchunk + c) * FIN_NV + k];
        vals[v][k] = s;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double Wt = 0.0, Et = 0.0, N0t = 0.0;
    for (int g = 0; g < G; g++) {
        Wt += S.accW[g];
        Et += S.accE[g];
        N0t += S.accN[(long long)g * L];
    }
    const double c0 = S.c[0];
    auto scal = [&](int v, double& e2, double& ev, double& a0) {
        double Wv = Wt - (v < G ? S.accW[v] : 0.0);
        double Ev = Et - (v < G ? S.accE[v] : 0.0);
        double N0v = N0t - (v < G ? S.accN[(long long)v * L] : 0.0);
        e2 = 0.0;
        for (int t = 0; t < MRQ_NTYPES; t++) e2 += vals[v][t * FIN_Q + 1];
        ev = Ev / Wv;
        a0 = c0 * c0 * N0v / Wv;
    };
    double e2f, evf, a0f;
    scal(G, e2f, evf, a0f);
    res->e0 = S.e0;
    res->e2 = e2f;
    res->e_var = evf;
    res->a0sq = a0f;
    res->e_mrci_q = evf + (1.0 - a0f) * (evf - S.e0);
    // jackknife
    double m_e2 = 0, m_ev = 0, m_a0 = 0, tn_m[MRQ_NTYPES], te_m[MRQ_NTYPES];
    for (int t = 0; t < MRQ_NTYPES; t++) tn_m[t] = te_m[t] = 0.0;
    for (int g = 0; g < G; g++) {
        double a, b, c;
        scal(g, a, b, c);
        m_e2 += a; m_ev += b; m_a0 += c;
        for (int t = 0; t < MRQ_NTYPES; t++) {
            tn_m[t] += vals[g][t * FIN_Q + 0];
            te_m[t] += vals[g][t * FIN_Q + 1];
        }
    }
    m_e2 /= G; m_ev /= G; m_a0 /= G;
    for (int t = 0; t < MRQ_NTYPES; t++) { tn_m[t] /= G; te_m[t] /= G; }
    double v_e2 = 0, v_ev = 0, v_a0 = 0, tn_v[MRQ_NTYPES], te_v[MRQ_NTYPES];
    for (int t = 0; t < MRQ_NTYPES; t++) tn_v[t] = te_v[t] = 0.0;
    for (int g = 0; g < G; g++) {
        double a, b, c;
        scal(g, a, b, c);
        v_e2 += (a - m_e2) * (a - m_e2);
        v_ev += (b - m_ev) * (b - m_ev);
        v_a0 += (c - m_a0) * (c - m_a0);
        for (int t = 0; t < MRQ_NTYPES; t++) {
            double x = vals[g][t * FIN_Q + 0] - tn_m[t], y = vals[g][t * FIN_Q + 1] - te_m[t];
            tn_v[t] += x * x;
            te_v[t] += y * y;
        }
    }
    const double f = G > 1 ? (double)(G - 1) / G : NAN;
    res->e2_sigma = sqrt(f * v_e2);
    res->e_var_sigma = sqrt(f * v_ev);
    res->a0sq_sigma = sqrt(f * v_a0);
    double scr_norm = 0.0, visited = 0.0;
    long long wsteps = 0;
    for (int t = 0; t < MRQ_NTYPES; t++) {
        res->type_norm[t] = vals[G][t * FIN_Q + 0];
        res->type_e2[t] = vals[G][t * FIN_Q + 1];
        res->type_screened[t] = vals[G][t * FIN_Q + 2];
        res->type_norm_sigma[t] = sqrt(f * tn_v[t]);
        res->type_e2_sigma[t] = sqrt(f * te_v[t]);
        scr_norm += vals[G][t * FIN_Q + 3];
        visited += vals[G][t * FIN_Q + 4];
        res->type_steps[t] = (long long)S.type_steps[t];
        wsteps += (long long)S.type_steps[t];
    }
    res->screened_norm = scr_norm;
    res->n_labels_visited = visited;
    res->walker_steps = wsteps;
}

// ============================================================================ SC-MRCI(s) optimisation (Eq. 8-9)

// grad[l] = (A_l - E B_l) / W over all groups, E = sum E / sum W: <delta_{l,l_n}/c_l (E_L - E)>
__global__ void k_mrci_grad(const SysDev* __restrict__ sys, double* __restrict__ grad, double* __restrict__ energy) {
    const SysDev S = *sys;
    double Wt = 0.0, Et = 0.0;
    for (int g = 0; g < S.G; g++) {
        Wt += S.accW[g];
        Et += S.accE[g];
    }
    const double E = Et / Wt;
    for (long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x; l < S.nlab; l += (long long)gridDim.x * blockDim.x) {
        double a = 0.0, b = 0.0;
        for (int g = 0; g < S.G; g++) {
            a += S.accA[(long long)g * S.nlab + l];
            b += S.accB[(long long)g * S.nlab + l];
        }
        grad[l] = (a - E * b) / Wt;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *energy = E;
}

// AMSGrad (Reddi, Kale, Kumar, ICLR 2018) on c_l, l >= 1; c_0 stays fixed (the energy does not
// depend on the overall scale of c)
__global__ void k_amsgrad(double* __restrict__ c, const double* __restrict__ g, double* __restrict__ m,
                          double* __restrict__ v, double* __restrict__ vh, long long nlab, double lr, double b1,
                          double b2, double eps) {
    for (long long l = 1 + (long long)blockIdx.x * blockDim.x + threadIdx.x; l < nlab; l += (long long)gridDim.x * blockDim.x) {
        const double gl = g[l];
        const double ml = b1 * m[l] + (1.0 - b1) * gl;
        const double vl = b2 * v[l] + (1.0 - b2) * gl * gl;
        const double vhl = fmax(vh[l], vl);
        m[l] = ml;
        v[l] = vl;
        vh[l] = vhl;
        c[l] -= lr * ml / (sqrt(vhl) + eps);
    }
}

// ============================================================================ fixed scratch for mrq_finalize_noalloc
//
// Partial sums of the finalize kernels for callers that cannot allocate device memory.  Every
// GPU that loads this library holds this array until the process exits.  All calls on a device
// share it: a call overwrites every slot it reads, and two calls whose kernels overlap on the
// GPU race on it.
static __device__ __align__(256) double g_noalloc_scratch[MRQ_NOALLOC_SCRATCH_DOUBLES];

#define MRQ_MAX_DEVICES 64
static double* g_noalloc_ptr[MRQ_MAX_DEVICES];     // device address of g_noalloc_scratch, per device
static std::mutex g_noalloc_mu;                    // guards g_noalloc_ptr (contexts may be created concurrently)

// device address of the fixed finalize scratch on `device` (current), looked up once per device
static double* noalloc_scratch_address(int device) {
    if (device < 0 || device >= MRQ_MAX_DEVICES) return nullptr;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_ptr[device] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) == cudaSuccess) g_noalloc_ptr[device] = (double*)p;
        else cudaGetLastError();
    }
    return g_noalloc_ptr[device];
}

// ============================================================================ host runtime

struct mrq_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    char err[1024] = {0};
    // Hamiltonian
    bool ham = false;
    int n = 0, nc = 0, na = 0, nv = 0, W = 1, nalpha = 0, nbeta = 0;
    double e_nuc = 0.0;
    long long neri = 0;
    double *d_h1 = nullptr, *d_eri = nullptr, *d_eri4 = nullptr, *d_tab = nullptr, *d_hc = nullptr,
           *d_eps = nullptr, *d_gamma = nullptr;
    unsigned short* d_colex = nullptr;
    long long nHs = 0, nPs = 0, nlab = 0;
    // reference
    bool ref = false;
    long long nref = 0;
    HashSlot* d_hash = nullptr;
    unsigned long long hcap = 0;
    unsigned long long start[4] = {0, 0, 0, 0};
    double start_c = 0.0;
    long long start_idx = 0;
    double e0 = 0, norm0 = 0, e_core = 0, sum_eps_core = 0;
    std::vector<double> eps, gamma;
    // coefficients
    double* d_c = nullptr;
    // walkers / accumulators
    Walker* d_walk = nullptr;
    long long nwalk = 0, walk_cap = 0;
    int G = 0;
    long long burn = 0;
    unsigned long long seed = 0;
    double tau = 1e-10;
    double *d_accN = nullptr, *d_accU = nullptr, *d_accW = nullptr, *d_accE = nullptr;
    double *d_accA = nullptr, *d_accB = nullptr;        // SC-MRCI gradient sums [G][nlab]
    double *d_grad = nullptr, *d_am_m = nullptr, *d_am_v = nullptr, *d_am_vh = nullptr;   // AMSGrad state
    unsigned long long* d_types = nullptr;
    long long acc_lab = 0;
    int acc_G = 0;
    int* d_err = nullptr;
    Walker** d_wptr = nullptr;                   // this context's walk set: one walker array
    Walker* h_wset_ptr = nullptr;                // (host staging of the copies above)
    long long h_wset_off[2] = {0, 0};
    long long* d_woff = nullptr;
    // batch tables (a batch launched through this context as the first of its list)
    SysDev* d_bsys = nullptr;
    Walker** d_bwptr = nullptr;
    long long* d_boff = nullptr;
    int bcap = 0;
    unsigned long long* d_sort_keys = nullptr;   // walker-slot ordering by determinant
    unsigned* d_sort_idx = nullptr;
    long long sort_cap = 0;
    size_t sort_smem = 0;
    double* d_partial = nullptr;
    long long partial_cap = 0;
    mrq_result* d_res = nullptr;
    SysDev hsys{};
    SysDev* d_sys = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // launch configuration (mrq_set_launch, mrq_tune_batch)
    int wpb = 0;                     // warps per walker block (0: chosen from the system's work units)
    int max_nw = MRQ_MAXNW;          // most warps per walker whose candidate lists fit shared memory
    int spl = 0;                     // steps per launch (0: every advance is one launch)
    int use_graph = 0;               // batches replay one reporting interval from a CUDA graph
    struct GraphKey {
        const void *sys = nullptr, *wptr = nullptr, *off = nullptr, *keys = nullptr;
        long long nslots = 0;
        int k = 0, wpb = 0, spl = 0, cap = 0, gstride = 0;
        bool operator==(const GraphKey& o) const {
            return sys == o.sys && wptr == o.wptr && off == o.off && keys == o.keys && nslots == o.nslots &&
                   k == o.k && wpb == o.wpb && spl == o.spl && cap == o.cap && gstride == o.gstride;
        }
    };
    // per determinant width, warps per walker (8, 4, 2, 1) and occupancy class (resident walk blocks
    // per SM, 4-1) of a batch launch
    static constexpr int NSLOT = 32;
    cudaGraphExec_t gexec[NSLOT] = {};
    GraphKey gkey[NSLOT];
    int smem_sm = 0, smem_rsv = 0;   // shared memory per SM and reserved per block (bytes)
    long long graph_replays = 0;
    long long* d_nbpre = nullptr;    // debug records: neighbour offsets of a determinant's units
    long long nbpre_cap = 0;
    Walker* d_tune = nullptr;        // the tuner's scratch copy of a batch's walkers
    long long tune_cap = 0;
    Walker** d_tptr = nullptr;
    int tptr_cap = 0;
    std::vector<cudaEvent_t> evs;    // start/stop pairs of the walk launches since the last finalize
    int launches = 0;
    long long launches_total = 0;
    double walk_ms = 0.0;
    long long total_steps = 0;
    // failure detection: host-wait deadline and lowered device bounds (mrq_set_deadline,
    // mrq_debug_set_limits)
    double deadline_s = 0.0;         // 0: host waits have no deadline
    cudaEvent_t ev_wait = nullptr;
    int probe_limit = 0, cap_limit = 0;
    int cand_cap_full = 1;           // the candidate-list capacity the loaded system needs
    double l2_fraction = 0.0;        // mrq_set_l2_window: share of the persisting-L2 carve-out for the tables
    int walk_minb = 2;               // resident walk blocks per SM of the kernel build in use (2, 3, 4)
};

static int fail(mrq_ctx* c, int code, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof c->err, fmt, ap);
        va_end(ap);
    }
    return code;
}

#define CK(call)                                                                                      \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? MRQ_OOM : MRQ_CUDA_ERROR, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                           \
    } while (0)

// Wait for the context stream.  With a deadline set (mrq_set_deadline) the wait polls an event
// and gives up with MRQ_DEVICE_TIMEOUT once the deadline passes; the device work keeps running
// and the next wait on this context waits for it again.
static int sync_stream(mrq_ctx* ctx) {
    if (!(ctx->deadline_s > 0.0) || ctx->ev_wait == nullptr) {
        CK(cudaStreamSynchronize(ctx->stream));
        return 0;
    }
    CK(cudaEventRecord(ctx->ev_wait, ctx->stream));
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaEventQuery(ctx->ev_wait);
        if (e == cudaSuccess) return 0;
        if (e != cudaErrorNotReady) return fail(ctx, MRQ_CUDA_ERROR, "cudaEventQuery: %s", cudaGetErrorString(e));
        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (dt > ctx->deadline_s)
            return fail(ctx, MRQ_DEVICE_TIMEOUT,
                        "device work did not finish within the %.6f s deadline; it keeps running and the next "
                        "call on this context waits for it", ctx->deadline_s);
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

// Set-up calls wait for earlier work under the deadline, then run their own kernels and copies to
// the end without one (so a timeout never leaves a half-built table or a temporary buffer behind).
struct DeadlinePause {
    mrq_ctx* c;
    double d;
    explicit DeadlinePause(mrq_ctx* ctx) : c(ctx), d(ctx->deadline_s) { ctx->deadline_s = 0.0; }
    ~DeadlinePause() { c->deadline_s = d; }
};

template <typename T>
static void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

static void free_reference(mrq_ctx* c) {
    dfree(c->d_hash);
    dfree(c->d_c);
    c->ref = false;
}
static void free_walkers(mrq_ctx* c) {
    dfree(c->d_walk);
    dfree(c->d_accN);
    dfree(c->d_accU);
    dfree(c->d_accA);
    dfree(c->d_accB);
    dfree(c->d_grad);
    dfree(c->d_am_m);
    dfree(c->d_am_v);
    dfree(c->d_am_vh);
    dfree(c->d_accW);
    dfree(c->d_accE);
    dfree(c->d_types);
    dfree(c->d_partial);
    c->nwalk = c->walk_cap = 0;
    c->acc_lab = 0;
    c->acc_G = 0;
    c->partial_cap = 0;
}
static void free_hamiltonian(mrq_ctx* c) {
    dfree(c->d_h1);
    dfree(c->d_eri);
    dfree(c->d_eri4);
    dfree(c->d_tab);
    dfree(c->d_hc);
    dfree(c->d_eps);
    dfree(c->d_gamma);
    dfree(c->d_colex);
    c->ham = false;
}

static int push_sys(mrq_ctx* ctx) {
    SysDev& s = ctx->hsys;
    s.accN = ctx->d_accN;
    s.accU = ctx->d_accU;
    s.accA = ctx->d_accA;
    s.accB = ctx->d_accB;
    s.accW = ctx->d_accW;
    s.accE = ctx->d_accE;
    s.type_steps = ctx->d_types;
    s.G = ctx->G;
    s.burn_in = ctx->burn;
    s.seed = ctx->seed;
    s.err = ctx->d_err;
    s.c = ctx->d_c;
    s.hash = ctx->d_hash;
    s.hmask = ctx->hcap ? ctx->hcap - 1 : 0;
    s.e0 = ctx->e0;
    s.e_core = ctx->e_core;
    s.sum_eps_core = ctx->sum_eps_core;
    s.max_probe = ctx->probe_limit > 0 ? std::min(64, ctx->probe_limit) : 64;
    s.cand_cap = ctx->cap_limit > 0 ? std::min(ctx->cand_cap_full, ctx->cap_limit) : ctx->cand_cap_full;
    CK(cudaMemcpyAsync(ctx->d_sys, &s, sizeof(SysDev), cudaMemcpyHostToDevice, ctx->stream));
    return 0;
}

static int check_err_flag(mrq_ctx* ctx, int* flag_out) {
    int f = 0;
    if (int r = sync_stream(ctx)) return r;
    CK(cudaMemcpyAsync(&f, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));    // idle already: returns at once
    *flag_out = f;
    return 0;
}

// launch-time options of a walk: warps (walkers) per block, whether to accumulate, and whether the
// one-time set-up (buffer growth, function attributes) has been done already (inside a stream capture)
struct WalkLaunch {
    int wpb = 8;
    int accumulate = 1;
    bool captured = false;
    cudaAccessPolicyWindow l2win = {};   // num_bytes 0: no persisting-L2 window
};

// scratch and shared memory of the per-system slot sort; max_seg = the most slots of one system
static int walk_sort_prepare(mrq_ctx* ctx, long long nslots, long long max_seg) {
    if (nslots > ctx->sort_cap) {
        dfree(ctx->d_sort_keys);
        dfree(ctx->d_sort_idx);
        CK(cudaMalloc(&ctx->d_sort_keys, sizeof(unsigned long long) * nslots));
        CK(cudaMalloc(&ctx->d_sort_idx, sizeof(unsigned) * nslots));
        ctx->sort_cap = nslots;
    }
    long long npad = 64;
    while (npad < std::min<long long>(max_seg, MRQ_SORT_MAX)) npad <<= 1;
    const size_t ssm = (size_t)npad * (sizeof(unsigned long long) + sizeof(unsigned));
    CK(cudaFuncSetAttribute(k_sort_slots, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm));
    ctx->sort_smem = ssm;
    return 0;
}

template <int W, int B>
static int walk_fits(mrq_ctx* ctx, size_t smem, int threads, bool& fits) {
    CK(cudaFuncSetAttribute(k_walk2<W, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int nb = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_walk2<W, B>, threads, smem));
    fits = nb >= B;
    return 0;
}

// the walk kernel's build for this launch: the most resident blocks per SM (4, 3 or 2, fewer
// registers each) that the block's shared memory allows
static int walk_attr_prepare(mrq_ctx* ctx, int W, size_t smem, int threads) {
    bool f4 = false, f3 = false, f2 = false;
    if (W == 1) {
        if (int r = walk_fits<1, 4>(ctx, smem, threads, f4)) return r;
        if (int r = walk_fits<1, 3>(ctx, smem, threads, f3)) return r;
        if (int r = walk_fits<1, 2>(ctx, smem, threads, f2)) return r;
    } else {
        if (int r = walk_fits<2, 2>(ctx, smem, threads, f2)) return r;
    }
    ctx->walk_minb = f4 ? 4 : (f3 ? 3 : 2);
    return 0;
}

// warps per walker block when the caller leaves the choice to the library: enough warps to share a
// CAS walker's work units, fewer for small systems whose units would leave warps idle
static int auto_warps(const SysDev& s) {
    const int u = s.unit_off[8];
    return u >= 512 ? 8 : (u >= 128 ? 4 : 2);
}
// warps per walker of a context's launches: the requested (or automatic) number, at most the most
// whose per-warp candidate lists fit shared memory (large active spaces run with fewer warps)
static int warps_of(const mrq_ctx* ctx) {
    return std::min(ctx->wpb > 0 ? ctx->wpb : auto_warps(ctx->hsys), ctx->max_nw);
}

// nsteps walker steps of a walk set: per step, order the slots by determinant (when the slot count
// allows a one-block sort), one block of L.wpb warps per walker slot (k_walk2), then the
// deterministic accumulation of the step's records (k_accum); `ctx` provides the stream and the
// sort scratch.  cap / gstride: the largest candidate-list capacity and single-operator size of
// the set's systems.
static int launch_walk(mrq_ctx* ctx, int W, const WalkSet& ws, int nsteps, int cap, int gstride,
                       const WalkLaunch& L = WalkLaunch()) {
    const int nw = std::min(L.wpb, MRQ_MAXNW);
    const size_t smem = cta_smem_bytes(nw, cap, gstride);
    const long long nslots = ws.nslots;
    if (!L.captured) {
        if (int r = walk_sort_prepare(ctx, nslots, ws.max_seg)) return r;
        if (int r = walk_attr_prepare(ctx, W, smem, 32 * nw)) return r;
    }
    for (int step = 0; step < nsteps; step++) {
        // order every system's slots by determinant (walkers on one determinant in neighbouring blocks)
        const unsigned nb = (unsigned)((nslots + 255) / 256);
        if (W == 1) k_walker_keys<1><<<nb, 256, 0, ctx->stream>>>(ws, ctx->d_sort_keys);
        else k_walker_keys<2><<<nb, 256, 0, ctx->stream>>>(ws, ctx->d_sort_keys);
        k_sort_slots<<<(unsigned)ws.nsys, 1024, ctx->sort_smem, ctx->stream>>>(ctx->d_sort_keys, ws.offsets,
                                                                              ctx->d_sort_idx);
        CK(cudaGetLastError());
        const unsigned* order = ctx->d_sort_idx;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)nslots);
        cfg.blockDim = dim3(32 * nw);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = ctx->stream;
        cudaLaunchAttribute attr[1];
        if (L.l2win.num_bytes > 0) {            // keep the walk's hottest table resident in L2
            attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
            attr[0].val.accessPolicyWindow = L.l2win;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
        }
        if (W == 2) CK(cudaLaunchKernelEx(&cfg, k_walk2<2, 2>, ws, order, L.accumulate));
        else if (ctx->walk_minb == 4) CK(cudaLaunchKernelEx(&cfg, k_walk2<1, 4>, ws, order, L.accumulate));
        else if (ctx->walk_minb == 3) CK(cudaLaunchKernelEx(&cfg, k_walk2<1, 3>, ws, order, L.accumulate));
        else CK(cudaLaunchKernelEx(&cfg, k_walk2<1, 2>, ws, order, L.accumulate));
        if (L.accumulate) {
            k_accum<<<dim3((unsigned)ws.nsys, 2), 1024, 0, ctx->stream>>>(ws);
            CK(cudaGetLastError());
        }
    }
    return 0;
}

// ---------------------------------------------------------------- work plan of the walk (host)

static long long nsub_h(long long k, int size) {
    if (size < 0 || k < size) return 0;
    return size == 0 ? 1 : (size == 1 ? k : k * (k - 1) / 2);
}
static long long shape_h(long long m, int cnt, int nal) {
    if (cnt == 0) return 1;
    if (cnt == 1) return m;
    return nal == 1 ? m * m : m * (m - 1) / 2;
}
// neighbours of one (X_a, Y_a) pair of a CAS walker with alpha(Y_a) - alpha(X_a) = d
static long long pair_total_h(int nc, int nv, int ka, int kb, int d) {
    long long tot = 0;
    for (int r = std::max(1, std::max(ka, kb)); r <= 2; r++) {
        const int c = r - ka, v = r - kb;
        if (c == 0 && v == 0) continue;
        for (int sc = 0; sc <= c; sc++) {
            const int sv = sc - d;
            if (sv < 0 || sv > v) continue;
            tot += shape_h(nc, c, sc) * shape_h(nv, v, sv);
        }
    }
    return tot;
}

// The CAS walkers' work units (the same for every CAS determinant: all hold n_alpha - n_core alpha
// and n_beta - n_core beta active electrons), the largest candidate list of a group (spin-resolved:
// the alpha count of R' fixes that of A'), and the walk block's shared memory.
static int walk_plan(mrq_ctx* ctx, SysDev& s) {
    const int nc = s.nc, na = s.na, nv = s.nv;
    const int nao = s.nalpha - nc, nbo = s.nbeta - nc, cea = na - nao, ceb = na - nbo;
    const int cntO = nao + nbo, cntE = cea + ceb;
    long long cas_nb = nao * (long long)cea + nbo * (long long)ceb + nsub_h(nao, 2) * nsub_h(cea, 2) +
                       nsub_h(nbo, 2) * nsub_h(ceb, 2) + (long long)nao * cea * nbo * ceb;
    long long total = cas_nb;
    long long off = (cas_nb + MRQ_CAS_CH - 1) / MRQ_CAS_CH;
    s.cas_nb = (int)cas_nb;
    s.cas_units = (int)off;
    for (int k = 0; k < 8; k++) {
        const int ka = k / 3, kb = k % 3;
        const long long npairs = nsub_h(cntO, ka) * nsub_h(cntE, kb);
        long long maxN = 0;
        for (int xal = 0; xal <= ka; xal++)
            for (int yal = 0; yal <= kb; yal++) {
                const long long nx = nsub_h(nao, xal) * nsub_h(nbo, ka - xal);
                const long long ny = nsub_h(cea, yal) * nsub_h(ceb, kb - yal);
                if (nx == 0 || ny == 0) continue;
                const long long N = pair_total_h(nc, nv, ka, kb, yal - xal);
                total += nx * ny * N;
                maxN = std::max(maxN, N);
            }
        const long long nch = std::max(1LL, (maxN + MRQ_UNIT_NB - 1) / MRQ_UNIT_NB);
        s.nch[k] = (int)nch;
        s.unit_off[k] = (int)off;
        off += npairs * nch;
    }
    s.unit_off[8] = (int)off;
    s.cas_nb_total = total;
    if (off > (1LL << 30) || total > (1LL << 40))
        return fail(ctx, MRQ_TOO_LARGE, "active space too large for the walk's work plan");
    // largest candidate list: m's active occupation differs from n's by at most two electrons
    long long cap = 1;
    for (int oa = std::max(0, nao - 2); oa <= std::min(na, nao + 2); oa++)
        for (int ob = std::max(0, nbo - 2); ob <= std::min(na, nbo + 2); ob++) {
            if (std::abs(oa + ob - cntO) > 2) continue;
            const int ea = na - oa, eb = na - ob;
            for (int c = 0; c <= 2; c++)
                for (int v = 0; v <= 2; v++) {
                    if (c == 0 && v == 0) continue;
                    for (int sc = 0; sc <= c; sc++)
                        for (int sv = 0; sv <= v; sv++) {
                            long long t = 0;
                            for (int rr = 1; rr <= 2; rr++) {
                                if (rr == 1 && (c > 1 || v > 1)) continue;
                                const int ne = rr - v, nf = rr - c;
                                if (ne < 0 || nf < 0) continue;
                                for (int i = 0; i <= ne; i++) {
                                    const int j = i + sv - sc;
                                    if (j < 0 || j > nf) continue;
                                    t += nsub_h(oa, i) * nsub_h(ob, ne - i) * nsub_h(ea, j) * nsub_h(eb, nf - j);
                                }
                            }
                            cap = std::max(cap, t);
                        }
                }
        }
    s.gstride = 2 * s.nca * s.nav;
    s.cand_cap = (int)cap;
    ctx->cand_cap_full = (int)cap;
    // the most warps per walker (8, 4, 2 or 1) whose candidate lists and operator fit one block's
    // shared memory; beyond one warp the active space is too large for the walk
    ctx->max_nw = 0;
    for (int nw = MRQ_MAXNW; nw >= 1 && ctx->max_nw == 0; nw >>= 1)
        if (cta_smem_bytes(nw, (int)cap, s.gstride) <= 227 * 1024) ctx->max_nw = nw;
    if (ctx->max_nw == 0)
        return fail(ctx, MRQ_TOO_LARGE, "active space too large for the shared-memory candidate lists");
    return 0;
}

// The persisting-L2 window of a walk launch (mrq_set_l2_window): the physicists' tables, which
// every reach-back term reads, marked persisting up to the device's carve-out (the carve-out is a
// per-process limit of this CUDA context and ends with it).
static int l2_window(mrq_ctx* ctx, cudaAccessPolicyWindow& w) {
    w = cudaAccessPolicyWindow{};
    if (!(ctx->l2_fraction > 0.0) || !ctx->d_tab) return 0;
    int maxwin = 0, maxpersist = 0;
    CK(cudaDeviceGetAttribute(&maxwin, cudaDevAttrMaxAccessPolicyWindowSize, ctx->device));
    CK(cudaDeviceGetAttribute(&maxpersist, cudaDevAttrMaxPersistingL2CacheSize, ctx->device));
    if (maxwin <= 0 || maxpersist <= 0) return 0;
    const size_t tab_bytes = sizeof(double) * 2 * (size_t)ctx->hsys.tab_half;
    const size_t carve = (size_t)(ctx->l2_fraction * (double)maxpersist);
    CK(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, carve));
    w.base_ptr = ctx->d_tab;
    w.num_bytes = std::min(tab_bytes, (size_t)maxwin);
    w.hitRatio = (float)std::min(1.0, (double)carve / (double)w.num_bytes);
    w.hitProp = cudaAccessPropertyPersisting;
    w.missProp = cudaAccessPropertyStreaming;
    return 0;
}

extern "C" {

int mrq_create(mrq_ctx** out, int device) {
    if (!out) return MRQ_INVALID_ARG;
    *out = nullptr;
    mrq_ctx* ctx = new mrq_ctx();
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        delete ctx;
        return MRQ_CUDA_ERROR;
    }
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&ctx->d_err, sizeof(int)) != cudaSuccess || cudaMalloc(&ctx->d_sys, sizeof(SysDev)) != cudaSuccess ||
        cudaMalloc(&ctx->d_res, sizeof(mrq_result)) != cudaSuccess || cudaEventCreate(&ctx->ev0) != cudaSuccess ||
        cudaEventCreate(&ctx->ev1) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_wait, cudaEventDisableTiming) != cudaSuccess) {
        mrq_destroy(ctx);
        return MRQ_CUDA_ERROR;
    }
    ctx->own_stream = true;
    cudaMemset(ctx->d_err, 0, sizeof(int));
    if (cudaDeviceGetAttribute(&ctx->smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, device) != cudaSuccess) {
        mrq_destroy(ctx);
        return MRQ_CUDA_ERROR;
    }
    // set-up of the allocation-free finalize: the device address of the fixed scratch array,
    // looked up once per device with that device current (host code cannot use the symbol itself)
    noalloc_scratch_address(device);
    *out = ctx;
    return 0;
}

void mrq_destroy(mrq_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_walkers(ctx);
    free_reference(ctx);
    free_hamiltonian(ctx);
    dfree(ctx->d_err);
    dfree(ctx->d_sys);
    dfree(ctx->d_res);
    dfree(ctx->d_sort_keys);
    dfree(ctx->d_sort_idx);
    dfree(ctx->d_wptr);
    dfree(ctx->d_woff);
    dfree(ctx->d_bsys);
    dfree(ctx->d_bwptr);
    dfree(ctx->d_boff);
    dfree(ctx->d_tune);
    dfree(ctx->d_tptr);
    dfree(ctx->d_nbpre);
    for (int w = 0; w < mrq_ctx::NSLOT; w++)
        if (ctx->gexec[w]) cudaGraphExecDestroy(ctx->gexec[w]);
    for (auto e : ctx->evs) cudaEventDestroy(e);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->ev_wait) cudaEventDestroy(ctx->ev_wait);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char* mrq_last_error(const mrq_ctx* ctx) { return ctx ? ctx->err : "null context"; }

int mrq_set_stream(mrq_ctx* ctx, void* stream) {
    if (!ctx) return MRQ_INVALID_ARG;
    CK(cudaSetDevice(ctx->device));
    if (int r_ = sync_stream(ctx)) return r_;
    if (stream) {
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        ctx->stream = (cudaStream_t)stream;
        ctx->own_stream = false;
    } else if (!ctx->own_stream) {
        CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
    }
    return 0;
}

int64_t mrq_n_labels(const mrq_ctx* ctx) { return (ctx && ctx->ham) ? ctx->nlab : 0; }

int mrq_load_hamiltonian(mrq_ctx* ctx, int n_core, int n_act, int n_virt, int n_alpha, int n_beta, const double* h1,
                         const double* eri, double e_core) {
    if (!ctx) return MRQ_INVALID_ARG;
    ctx->err[0] = 0;
    const int n = n_core + n_act + n_virt;
    if (n_core < 0 || n_act < 0 || n_virt < 0 || n <= 0 || n > MRQ_MAXN || n_core > 64 || n_act > 32 || !h1 ||
        !eri)
        return fail(ctx, MRQ_INVALID_ARG, "orbital counts out of range (n <= 128, n_core <= 64, n_act <= 32)");
    if (n_alpha < n_core || n_beta < n_core || n_alpha > n_core + n_act || n_beta > n_core + n_act)
        return fail(ctx, MRQ_INVALID_ARG, "electron counts must fill the core and fit the active space");
    CK(cudaSetDevice(ctx->device));
    if (int r_ = sync_stream(ctx)) return r_;
    DeadlinePause pause_(ctx);
    free_walkers(ctx);
    free_reference(ctx);
    free_hamiltonian(ctx);
    ctx->n = n;
    ctx->nc = n_core;
    ctx->na = n_act;
    ctx->nv = n_virt;
    ctx->W = (n + 63) / 64;
    ctx->nalpha = n_alpha;
    ctx->nbeta = n_beta;
    ctx->e_nuc = e_core;
    const long long npair = (long long)n * (n + 1) / 2;
    ctx->neri = npair * (npair + 1) / 2;
    ctx->nHs = 1 + 2LL * n_core + (2LL * n_core) * (2LL * n_core - 1) / 2;
    ctx->nPs = 1 + 2LL * n_virt + (2LL * n_virt) * (2LL * n_virt - 1) / 2;
    ctx->nlab = ctx->nHs * ctx->nPs;
    CK(cudaMalloc(&ctx->d_h1, sizeof(double) * n * n));
    CK(cudaMalloc(&ctx->d_eri, sizeof(double) * ctx->neri));
    CK(cudaMalloc(&ctx->d_eri4, sizeof(double) * npair * n * n));
    const long long nca = n_core + n_act, nav = n_act + n_virt;
    CK(cudaMalloc(&ctx->d_tab, sizeof(double) * 2 * std::max(1LL, nca * nca * nav * nav)));
    CK(cudaMalloc(&ctx->d_hc, sizeof(double) * n * n));
    CK(cudaMalloc(&ctx->d_eps, sizeof(double) * n));
    CK(cudaMalloc(&ctx->d_gamma, sizeof(double) * std::max(1, n_act * n_act)));
    {
        // co-lexicographic pair table of up to 128 items: colex[j(j-1)/2 + i] = i | j << 8, i < j
        std::vector<unsigned short> colex(128 * 127 / 2);
        for (int j = 1, q = 0; j < 128; j++)
            for (int i = 0; i < j; i++) colex[q++] = (unsigned short)(i | (j << 8));
        CK(cudaMalloc(&ctx->d_colex, sizeof(unsigned short) * colex.size()));
        CK(cudaMemcpyAsync(ctx->d_colex, colex.data(), sizeof(unsigned short) * colex.size(), cudaMemcpyHostToDevice,
                           ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    CK(cudaMemcpyAsync(ctx->d_h1, h1, sizeof(double) * n * n, cudaMemcpyDefault, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_eri, eri, sizeof(double) * ctx->neri, cudaMemcpyDefault, ctx->stream));
    SysDev& s = ctx->hsys;
    s = SysDev{};
    s.n = n;
    s.nc = n_core;
    s.na = n_act;
    s.nv = n_virt;
    s.W = ctx->W;
    s.nalpha = n_alpha;
    s.nbeta = n_beta;
    s.nPs = ctx->nPs;
    s.nlab = ctx->nlab;
    for (int w = 0; w < 2; w++) {
        s.mcore[w] = s.mact[w] = s.mvirt[w] = 0;
        for (int q = 64 * w; q < 64 * w + 64 && q < n; q++) {
            unsigned long long b = 1ull << (q - 64 * w);
            if (q < n_core) s.mcore[w] |= b;
            else if (q < n_core + n_act) s.mact[w] |= b;
            else s.mvirt[w] |= b;
        }
    }
    s.eri = ctx->d_eri;
    s.eri4 = ctx->d_eri4;
    s.tab = ctx->d_tab;
    s.nca = (int)nca;
    s.nav = (int)nav;
    s.tab_half = (unsigned)(nca * nca * nav * nav);
    s.colex = ctx->d_colex;
    s.mag_c = n_core > 1 ? ~0ull / (unsigned long long)n_core + 1ull : 0ull;
    s.mag_v = n_virt > 1 ? ~0ull / (unsigned long long)n_virt + 1ull : 0ull;
    s.h1 = ctx->d_h1;
    s.hc = ctx->d_hc;
    s.eps = ctx->d_eps;
    s.e_nuc = e_core;
    s.max_probe = 64;
    s.G = 1;
    if (int r = walk_plan(ctx, s)) return r;
    if (int r = push_sys(ctx)) return r;
    k_expand_eri<<<1216, 256, 0, ctx->stream>>>(ctx->d_eri, ctx->d_eri4, n);
    CK(cudaGetLastError());
    k_build_tab<<<2432, 256, 0, ctx->stream>>>(ctx->d_sys, ctx->d_tab);
    CK(cudaGetLastError());
    k_core_fock<<<(n * n + 127) / 128, 128, 0, ctx->stream>>>(ctx->d_sys, ctx->d_hc);
    CK(cudaGetLastError());
    if (int r_ = sync_stream(ctx)) return r_;
    ctx->ham = true;
    return 0;
}

int mrq_load_reference(mrq_ctx* ctx, int64_t n_det, const uint64_t* dets, const double* coeffs) {
    if (!ctx) return MRQ_INVALID_ARG;
    ctx->err[0] = 0;
    if (!ctx->ham) return fail(ctx, MRQ_NOT_LOADED, "load the Hamiltonian first");
    if (n_det <= 0 || !dets || !coeffs) return fail(ctx, MRQ_INVALID_ARG, "empty reference");
    CK(cudaSetDevice(ctx->device));
    if (int r_ = sync_stream(ctx)) return r_;
    DeadlinePause pause_(ctx);
    free_walkers(ctx);
    free_reference(ctx);
    const int W = ctx->W;
    unsigned long long cap = 16;
    while (cap < 4ull * (unsigned long long)n_det) cap <<= 1;
    ctx->hcap = cap;
    ctx->nref = n_det;
    unsigned long long* d_dets = nullptr;
    double* d_co = nullptr;
    CK(cudaMalloc(&ctx->d_hash, sizeof(HashSlot) * cap));
    CK(cudaMalloc(&d_dets, sizeof(unsigned long long) * 2 * W * n_det));
    CK(cudaMalloc(&d_co, sizeof(double) * n_det));
    CK(cudaMalloc(&ctx->d_c, sizeof(double) * ctx->nlab));
    CK(cudaMemcpyAsync(d_dets, dets, sizeof(unsigned long long) * 2 * W * n_det, cudaMemcpyDefault, ctx->stream));
    CK(cudaMemcpyAsync(d_co, coeffs, sizeof(double) * n_det, cudaMemcpyDefault, ctx->stream));
    {
        std::vector<double> c(ctx->nlab, 0.1);
        c[0] = 1.0;
        CK(cudaMemcpyAsync(ctx->d_c, c.data(), sizeof(double) * ctx->nlab, cudaMemcpyHostToDevice, ctx->stream));
        if (int r_ = sync_stream(ctx)) return r_;
    }
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    if (int r = push_sys(ctx)) return r;
    k_hash_clear<<<(unsigned)((cap + 255) / 256), 256, 0, ctx->stream>>>(ctx->d_hash, cap);
    const unsigned nbk = (unsigned)((n_det + 127) / 128);
    if (W == 1) k_hash_build<1><<<nbk, 128, 0, ctx->stream>>>(ctx->d_sys, ctx->d_hash, d_dets, d_co, n_det, ctx->d_err);
    else k_hash_build<2><<<nbk, 128, 0, ctx->stream>>>(ctx->d_sys, ctx->d_hash, d_dets, d_co, n_det, ctx->d_err);
    CK(cudaGetLastError());
    int flag = 0;
    if (int r = check_err_flag(ctx, &flag)) return r;
    if (flag) {
        cudaFree(d_dets);
        cudaFree(d_co);
        free_reference(ctx);
        if (flag & 32) return fail(ctx, MRQ_HASH_OVERFLOW, "hash insertion ran past the probe bound");
        return fail(ctx, MRQ_BAD_REFERENCE, "reference determinant with a core hole, a virtual electron, "
                                            "a wrong electron count or a duplicate (flags %d)", flag);
    }
    // start determinant: largest |c| (first on ties)
    long long* d_idx = nullptr;
    CK(cudaMalloc(&d_idx, sizeof(long long)));
    k_argmax_abs<<<1, 1024, 0, ctx->stream>>>(d_co, n_det, d_idx);
    CK(cudaMemcpyAsync(&ctx->start_idx, d_idx, sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream));
    if (int r_ = sync_stream(ctx)) return r_;
    cudaFree(d_idx);
    memset(ctx->start, 0, sizeof ctx->start);
    {
        unsigned long long tmp[4] = {0, 0, 0, 0};
        CK(cudaMemcpy(tmp, d_dets + ctx->start_idx * 2 * W, sizeof(unsigned long long) * 2 * W, cudaMemcpyDeviceToHost));
        for (int w = 0; w < W; w++) {
            ctx->start[w] = tmp[w];
            ctx->start[2 + w] = tmp[W + w];
        }
        CK(cudaMemcpy(&ctx->start_c, d_co + ctx->start_idx, sizeof(double), cudaMemcpyDeviceToHost));
    }
    // E0, norm, gamma, eps
    const int nblk = 304;
    double* d_part = nullptr;
    double* d_scal = nullptr;
    CK(cudaMalloc(&d_part, sizeof(double) * 2 * nblk));
    CK(cudaMalloc(&d_scal, sizeof(double) * 8));
    if (W == 1) k_ref_energy<1><<<nblk, 128, 0, ctx->stream>>>(ctx->d_sys, d_dets, d_co, n_det, d_part);
    else k_ref_energy<2><<<nblk, 128, 0, ctx->stream>>>(ctx->d_sys, d_dets, d_co, n_det, d_part);
    CK(cudaGetLastError());
    if (ctx->na > 0) {
        if (W == 1) k_ref_rdm<1><<<ctx->na * ctx->na, 256, 0, ctx->stream>>>(ctx->d_sys, d_dets, d_co, n_det, ctx->d_gamma);
        else k_ref_rdm<2><<<ctx->na * ctx->na, 256, 0, ctx->stream>>>(ctx->d_sys, d_dets, d_co, n_det, ctx->d_gamma);
        CK(cudaGetLastError());
    }
    k_setup_finish<<<1, 256, 0, ctx->stream>>>(ctx->d_sys, d_part, nblk, ctx->d_gamma, ctx->d_eps, d_scal);
    CK(cudaGetLastError());
    double scal[8];
    CK(cudaMemcpyAsync(scal, d_scal, sizeof(double) * 4, cudaMemcpyDeviceToHost, ctx->stream));
    ctx->eps.assign(ctx->n, 0.0);
    ctx->gamma.assign((size_t)ctx->na * ctx->na, 0.0);
    CK(cudaMemcpyAsync(ctx->eps.data(), ctx->d_eps, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
    if (ctx->na)
        CK(cudaMemcpyAsync(ctx->gamma.data(), ctx->d_gamma, sizeof(double) * ctx->na * ctx->na, cudaMemcpyDeviceToHost,
                           ctx->stream));
    if (int r_ = sync_stream(ctx)) return r_;
    cudaFree(d_part);
    cudaFree(d_scal);
    cudaFree(d_dets);
    cudaFree(d_co);
    ctx->e0 = scal[0];
    ctx->norm0 = scal[1];
    ctx->e_core = scal[2];
    ctx->sum_eps_core = scal[3];
    int flag2 = 0;
    if (int r = check_err_flag(ctx, &flag2)) return r;
    if (flag2 & MRQ_ERR_HASH) return fail(ctx, MRQ_HASH_OVERFLOW, "hash probe bound exceeded during setup");
    if (int r = push_sys(ctx)) return r;
    if (int r_ = sync_stream(ctx)) return r_;
    ctx->ref = true;
    return 0;
}

int mrq_set_coeffs(mrq_ctx* ctx, int64_t n_labels, const double* c) {
    if (!ctx) return MRQ_INVALID_ARG;
    ctx->err[0] = 0;
    if (!ctx->ref) return fail(ctx, MRQ_NOT_LOADED, "load the Hamiltonian and the reference first");
    if (n_labels != ctx->nlab || !c)
        return fail(ctx, MRQ_INVALID_ARG, "expected %lld coefficients", (long long)ctx->nlab);
    CK(cudaSetDevice(ctx->device));
    dfree(ctx->d_am_m);     // a new coefficient vector starts a new optimisation
    dfree(ctx->d_am_v);
    dfree(ctx->d_am_vh);
    CK(cudaMemcpyAsync(ctx->d_c, c, sizeof(double) * n_labels, cudaMemcpyDefault, ctx->stream));
    if (int r_ = sync_stream(ctx)) return r_;
    return 0;
}

int mrq_setup_info(mrq_ctx* ctx, double* out5, double* eps, double* gamma) {
    if (!ctx || !out5) return MRQ_INVALID_ARG;
    if (!ctx->ref) return fail(ctx, MRQ_NOT_LOADED, "no reference loaded");
    out5[0] = ctx->e0;
    out5[1] = ctx->norm0;
    out5[2] = ctx->e_core;
    out5[3] = ctx->sum_eps_core;
    out5[4] = (double)ctx->start_idx;
    if (eps) memcpy(eps, ctx->eps.data(), sizeof(double) * ctx->n);
    if (gamma && ctx->na) memcpy(gamma, ctx->gamma.data(), sizeof(double) * ctx->na * ctx->na);
    return 0;
}

int mrq_debug_local(mrq_ctx* ctx, int64_t n, const uint64_t* dets, mrq_local* local, int64_t max_nb,
                    mrq_neighbour* nb) {
    if (!ctx) return MRQ_INVALID_ARG;
    ctx->err[0] = 0;
    if (!ctx->ref) return fail(ctx, MRQ_NOT_LOADED, "no reference loaded");
    if (n <= 0 || !dets || !local || (nb && max_nb <= 0)) return fail(ctx, MRQ_INVALID_ARG, "bad arguments");
    CK(cudaSetDevice(ctx->device));
    DeadlinePause pause_(ctx);
    const int W = ctx->W;
    unsigned long long* d_dets = nullptr;
    mrq_local* d_loc = nullptr;
    mrq_neighbour* d_nb = nullptr;
    CK(cudaMalloc(&d_dets, sizeof(unsigned long long) * 2 * W * n));
    CK(cudaMalloc(&d_loc, sizeof(mrq_local) * n));
    if (nb) CK(cudaMalloc(&d_nb, sizeof(mrq_neighbour) * n * max_nb));
    CK(cudaMemcpyAsync(d_dets, dets, sizeof(unsigned long long) * 2 * W * n, cudaMemcpyDefault, ctx->stream));
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    if (int r = push_sys(ctx)) return r;
    const int cap = ctx->hsys.cand_cap;
    const int nw = std::min(warps_of(ctx), MRQ_MAXNW);
    const size_t smem = cta_smem_bytes(nw, cap, ctx->hsys.gstride);
    // neighbour offsets of the CAS units, for the records
    const long long stride = nb ? std::max(1, ctx->hsys.unit_off[8]) : 0;
    if (nb && n * stride > ctx->nbpre_cap) {
        dfree(ctx->d_nbpre);
        CK(cudaMalloc(&ctx->d_nbpre, sizeof(long long) * n * stride));
        ctx->nbpre_cap = n * stride;
    }
    long long* pre = nb ? ctx->d_nbpre : nullptr;
    if (W == 1) {
        CK(cudaFuncSetAttribute(k_debug2<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_debug2<1><<<(unsigned)n, 32 * nw, smem, ctx->stream>>>(ctx->d_sys, d_dets, n, d_loc, max_nb, d_nb, pre,
                                                                 (int)stride);
    } else {
        CK(cudaFuncSetAttribute(k_debug2<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_debug2<2><<<(unsigned)n, 32 * nw, smem, ctx->stream>>>(ctx->d_sys, d_dets, n, d_loc, max_nb, d_nb, pre,
                                                                 (int)stride);
    }
    CK(cudaGetLastError());
    if (int r = sync_stream(ctx)) return r;
    CK(cudaMemcpyAsync(local, d_loc, sizeof(mrq_local) * n, cudaMemcpyDeviceToHost, ctx->stream));
    if (nb) CK(cudaMemcpyAsync(nb, d_nb, sizeof(mrq_neighbour) * n * max_nb, cudaMemcpyDeviceToHost, ctx->stream));
    int flag = 0;
    if (int r = check_err_flag(ctx, &flag)) return r;
    cudaFree(d_dets);
    cudaFree(d_loc);
    if (d_nb) cudaFree(d_nb);
    if (flag & MRQ_ERR_HASH) return fail(ctx, MRQ_HASH_OVERFLOW, "hash probe bound exceeded");
    if (flag & MRQ_ERR_CAP) return fail(ctx, MRQ_TOO_LARGE, "candidate list capacity exceeded");
    return 0;
}

int mrq_walkers_init(mrq_ctx* ctx, const mrq_sample_params* p) {
    if (!ctx || !p) return MRQ_INVALID_ARG;
    ctx->err[0] = 0;
    if (!ctx->ref) return fail(ctx, MRQ_NOT_LOADED, "no reference loaded");
    if (p->n_walkers <= 0 || p->n_groups <= 0 || p->n_groups > 64 || p->n_steps < 0 || p->burn_in < 0)
        return fail(ctx, MRQ_INVALID_ARG, "need n_walkers > 0, 1 <= n_groups <= 64, n_steps >= 0, burn_in >= 0");
    if (p->warps_per_walker != 0 && p->warps_per_walker != 1 && p->warps_per_walker != 2 && p->warps_per_walker != 4 &&
        p->warps_per_walker != 8)
        return fail(ctx, MRQ_INVALID_ARG, "warps_per_walker must be 0, 1, 2, 4 or 8");
    if (p->steps_per_check < 0 || p->target_sigma < 0.0)
        return fail(ctx, MRQ_INVALID_ARG, "need steps_per_check >= 0 and target_sigma >= 0");
    if (p->warps_per_walker) ctx->wpb = p->warps_per_walker;
    CK(cudaSetDevice(ctx->device));
    DeadlinePause pause_(ctx);
    if (p->n_walkers > ctx->walk_cap) {
        dfree(ctx->d_walk);
        CK(cudaMalloc(&ctx->d_walk, sizeof(Walker) * p->n_walkers));
        ctx->walk_cap = p->n_walkers;
    }
    if (ctx->acc_lab != ctx->nlab || ctx->acc_G != p->n_groups) {
        dfree(ctx->d_accN);
        dfree(ctx->d_accU);
        dfree(ctx->d_accW);
        dfree(ctx->d_accE);
        dfree(ctx->d_types);
        CK(cudaMalloc(&ctx->d_accN, sizeof(double) * ctx->nlab * p->n_groups));
        CK(cudaMalloc(&ctx->d_accU, sizeof(double) * ctx->nlab * p->n_groups));
        dfree(ctx->d_accA);
        dfree(ctx->d_accB);
        CK(cudaMalloc(&ctx->d_accA, sizeof(double) * ctx->nlab * p->n_groups));
        CK(cudaMalloc(&ctx->d_accB, sizeof(double) * ctx->nlab * p->n_groups));
        CK(cudaMalloc(&ctx->d_accW, sizeof(double) * p->n_groups));
        CK(cudaMalloc(&ctx->d_accE, sizeof(double) * p->n_groups));
        CK(cudaMalloc(&ctx->d_types, sizeof(unsigned long long) * MRQ_NTYPES));
        ctx->acc_lab = ctx->nlab;
        ctx->acc_G = p->n_groups;
    }
    ctx->nwalk = p->n_walkers;
    ctx->G = p->n_groups;
    ctx->burn = p->burn_in;
    ctx->seed = p->seed;
    ctx->tau = p->screen_tau;
    ctx->total_steps = 0;
    ctx->walk_ms = 0.0;
    ctx->launches = 0;
    ctx->launches_total = 0;
    CK(cudaMemsetAsync(ctx->d_accN, 0, sizeof(double) * ctx->nlab * ctx->G, ctx->stream));
    CK(cudaMemsetAsync(ctx->d_accU, 0, sizeof(double) * ctx->nlab * ctx->G, ctx->stream));
    CK(cudaMemsetAsync(ctx->d_accA, 0, sizeof(double) * ctx->nlab * ctx->G, ctx->stream));
    CK(cudaMemsetAsync(ctx->d_accB, 0, sizeof(double) * ctx->nlab * ctx->G, ctx->stream));
    CK(cudaMemsetAsync(ctx->d_accW, 0, sizeof(double) * ctx->G, ctx->stream));
    CK(cudaMemsetAsync(ctx->d_accE, 0, sizeof(double) * ctx->G, ctx->stream));
    CK(cudaMemsetAsync(ctx->d_types, 0, sizeof(unsigned long long) * MRQ_NTYPES, ctx->stream));
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    if (int r = push_sys(ctx)) return r;
    double c0 = 1.0;
    CK(cudaMemcpyAsync(&c0, ctx->d_c, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (int r_ = sync_stream(ctx)) return r_;
    if (!ctx->d_wptr) {
        CK(cudaMalloc(&ctx->d_wptr, sizeof(Walker*)));
        CK(cudaMalloc(&ctx->d_woff, 2 * sizeof(long long)));
    }
    {
        ctx->h_wset_ptr = ctx->d_walk;
        ctx->h_wset_off[0] = 0;
        ctx->h_wset_off[1] = ctx->nwalk;
        CK(cudaMemcpyAsync(ctx->d_wptr, &ctx->h_wset_ptr, sizeof(Walker*), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->d_woff, ctx->h_wset_off, 2 * sizeof(long long), cudaMemcpyHostToDevice, ctx->stream));
    }
    k_walkers_init<<<(unsigned)((ctx->nwalk + 255) / 256), 256, 0, ctx->stream>>>(
        ctx->d_walk, ctx->nwalk, ctx->start[0], ctx->start[1], ctx->start[2], ctx->start[3], c0 * ctx->start_c, 0, ctx->G);
    CK(cudaGetLastError());
    return 0;
}

int mrq_walkers_advance(mrq_ctx* ctx, int64_t n_steps) {
    if (!ctx) return MRQ_INVALID_ARG;
    if (!ctx->ref || !ctx->d_walk || ctx->nwalk == 0) return fail(ctx, MRQ_NOT_LOADED, "walkers not initialised");
    if (n_steps <= 0) return 0;
    CK(cudaSetDevice(ctx->device));
    const size_t k = (size_t)ctx->launches * 2;
    while (ctx->evs.size() < k + 2) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        ctx->evs.push_back(e);
    }
    CK(cudaEventRecord(ctx->evs[k], ctx->stream));
    WalkSet ws{ctx->d_sys, ctx->d_wptr, ctx->d_woff, 1, ctx->nwalk};
    ws.max_seg = ctx->nwalk;
    WalkLaunch L;
    L.wpb = warps_of(ctx);
    if (int r = l2_window(ctx, L.l2win)) return r;
    const int64_t spl = ctx->spl > 0 ? ctx->spl : n_steps;
    for (int64_t done = 0; done < n_steps; done += spl)
        if (int r = launch_walk(ctx, ctx->W, ws, (int)std::min<int64_t>(spl, n_steps - done), ctx->hsys.cand_cap,
                                ctx->hsys.gstride, L))
            return r;
    CK(cudaGetLastError());
    CK(cudaEventRecord(ctx->evs[k + 1], ctx->stream));
    ctx->launches++;
    ctx->total_steps += n_steps * ctx->nwalk;
    return 0;
}

static const long long FIN_CHUNK = 8192;

static long long fin_scratch_doubles(const mrq_ctx* ctx, int* nchunk) {
    *nchunk = (int)((ctx->nlab + FIN_CHUNK - 1) / FIN_CHUNK);
    return (long long)(ctx->G + 1) * (*nchunk) * FIN_NV;
}

// finalize with the partial sums in `scratch` (at least fin_scratch_doubles() doubles)
// (the device copy of the system is current since mrq_walkers_init pushed it, so nothing is copied
// in: a copy from pageable host memory would wait for the walk and defeat the deadline)
static int finalize_with(mrq_ctx* ctx, mrq_result* out, double* scratch, int nchunk) {
    k_fin_labels<<<(ctx->G + 1) * nchunk, 256, 0, ctx->stream>>>(ctx->d_sys, ctx->tau, nchunk, FIN_CHUNK, scratch);
    CK(cudaGetLastError());
    k_fin_reduce<<<1, 256, 0, ctx->stream>>>(ctx->d_sys, scratch, nchunk, ctx->d_res);
    CK(cudaGetLastError());
    if (int r = sync_stream(ctx)) return r;
    CK(cudaMemcpyAsync(out, ctx->d_res, sizeof(mrq_result), cudaMemcpyDeviceToHost, ctx->stream));
    int flag = 0;
    if (int r = check_err_flag(ctx, &flag)) return r;
    for (int i = 0; i < ctx->launches; i++) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, ctx->evs[2 * i], ctx->evs[2 * i + 1]) == cudaSuccess) ctx->walk_ms += ms;
    }
    out->walk_launches = ctx->launches_total += ctx->launches;
    ctx->launches = 0;
    out->seconds = ctx->walk_ms * 1e-3;
    out->total_steps = ctx->total_steps;
    out->status = 0;
    if (flag & MRQ_ERR_HASH) out->status = MRQ_HASH_OVERFLOW;
    else if (flag & MRQ_ERR_CAP) out->status = MRQ_TOO_LARGE;
    else if (flag & (MRQ_ERR_NOMOVE | MRQ_ERR_LABEL)) out->status = MRQ_NO_MOVE;
    if (out->status) return fail(ctx, out->status, "device flagged an error during the walk (flags %d)", flag);
    return 0;
}

int mrq_finalize(mrq_ctx* ctx, mrq_result* out) {
    if (!ctx || !out) return MRQ_INVALID_ARG;
    if (!ctx->ref || !ctx->d_accN) return fail(ctx, MRQ_NOT_LOADED, "walkers not initialised");
    CK(cudaSetDevice(ctx->device));
    int nchunk = 0;
    const long long need = fin_scratch_doubles(ctx, &nchunk);
    if (need > ctx->partial_cap) {
        dfree(ctx->d_partial);
        CK(cudaMalloc(&ctx->d_partial, sizeof(double) * need));
        ctx->partial_cap = need;
    }
    return finalize_with(ctx, out, ctx->d_partial, nchunk);
}

int mrq_finalize_noalloc(mrq_ctx* ctx, mrq_result* out) {
    if (!ctx || !out) return MRQ_INVALID_ARG;
    ctx->err[0] = 0;
    if (!ctx->ref || !ctx->d_accN) return fail(ctx, MRQ_NOT_LOADED, "walkers not initialised");
    double* scratch = nullptr;
    if (ctx->device >= 0 && ctx->device < MRQ_MAX_DEVICES) {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        scratch = g_noalloc_ptr[ctx->device];
    }
    if (scratch == nullptr)
        return fail(ctx, MRQ_CUDA_ERROR, "fixed finalize scratch has no device address on device %d", ctx->device);
    int nchunk = 0;
    const long long need = fin_scratch_doubles(ctx, &nchunk);
    if (need > MRQ_NOALLOC_SCRATCH_DOUBLES)
        return fail(ctx, MRQ_TOO_LARGE,
                    "mrq_finalize_noalloc: %lld labels x %d groups need %lld scratch doubles, more than its fixed "
                    "%d (use mrq_finalize)", (long long)ctx->nlab, ctx->G, need, MRQ_NOALLOC_SCRATCH_DOUBLES);
    CK(cudaSetDevice(ctx->device));
    return finalize_with(ctx, out, scratch, nchunk);
}

int mrq_mrci_gradient(mrq_ctx* ctx, double* grad, double* energy) {
    if (!ctx) return MRQ_INVALID_ARG;
    ctx->err[0] = 0;
    if (!ctx->ref || !ctx->d_accA) return fail(ctx, MRQ_NOT_LOADED, "no walk to take the gradient from");
    CK(cudaSetDevice(ctx->device));
    if (!ctx->d_grad) CK(cudaMalloc(&ctx->d_grad, sizeof(double) * (ctx->nlab + 1)));
    if (int r = push_sys(ctx)) return r;
    k_mrci_grad<<<(unsigned)std::min<long long>(1024, (ctx->nlab + 255) / 256), 256, 0, ctx->stream>>>(
        ctx->d_sys, ctx->d_grad, ctx->d_grad + ctx->nlab);
    CK(cudaGetLastError());
    double e = 0.0;
    if (grad) CK(cudaMemcpyAsync(grad, ctx->d_grad, sizeof(double) * ctx->nlab, cudaMemcpyDefault, ctx->stream));
    CK(cudaMemcpyAsync(&e, ctx->d_grad + ctx->nlab, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (int r_ = sync_stream(ctx)) return r_;
    if (energy) *energy = e;
    return 0;
}

int mrq_amsgrad_step(mrq_ctx* ctx, double lr, double beta1, double beta2, double eps) {
    if (!ctx) return MRQ_INVALID_ARG;
    ctx->err[0] = 0;
    if (!ctx->d_grad) return fail(ctx, MRQ_NOT_LOADED, "call mrq_mrci_gradient first");
    if (!(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
        return fail(ctx, MRQ_INVALID_ARG, "need lr > 0, 0 <= beta < 1, eps > 0");
    CK(cudaSetDevice(ctx->device));
    if (!ctx->d_am_m) {
        CK(cudaMalloc(&ctx->d_am_m, sizeof(double) * ctx->nlab));
        CK(cudaMalloc(&ctx->d_am_v, sizeof(double) * ctx->nlab));
        CK(cudaMalloc(&ctx->d_am_vh, sizeof(double) * ctx->nlab));
        CK(cudaMemsetAsync(ctx->d_am_m, 0, sizeof(double) * ctx->nlab, ctx->stream));
        CK(cudaMemsetAsync(ctx->d_am_v, 0, sizeof(double) * ctx->nlab, ctx->stream));
        CK(cudaMemsetAsync(ctx->d_am_vh, 0, sizeof(double) * ctx->nlab, ctx->stream));
    }
    k_amsgrad<<<(unsigned)std::min<long long>(1024, (ctx->nlab + 255) / 256), 256, 0, ctx->stream>>>(
        ctx->d_c, ctx->d_grad, ctx->d_am_m, ctx->d_am_v, ctx->d_am_vh, ctx->nlab, lr, beta1, beta2, eps);
    CK(cudaGetLastError());
    if (int r_ = sync_stream(ctx)) return r_;
    return 0;
}

int mrq_read_coeffs(mrq_ctx* ctx, double* c) {
    if (!ctx || !c) return MRQ_INVALID_ARG;
    if (!ctx->ref) return fail(ctx, MRQ_NOT_LOADED, "no reference loaded");
    CK(cudaSetDevice(ctx->device));
    if (int r = sync_stream(ctx)) return r;
    CK(cudaMemcpyAsync(c, ctx->d_c, sizeof(double) * ctx->nlab, cudaMemcpyDefault, ctx->stream));
    if (int r_ = sync_stream(ctx)) return r_;
    return 0;
}

static int batch_check(mrq_ctx* const* ctxs, int n) {
    if (!ctxs || n <= 0) return MRQ_INVALID_ARG;
    mrq_ctx* lead = ctxs[0];
    if (!lead) return MRQ_INVALID_ARG;
    for (int i = 0; i < n; i++) {
        if (!ctxs[i]) return fail(lead, MRQ_INVALID_ARG, "context %d is null", i);
        if (ctxs[i]->device != lead->device)
            return fail(lead, MRQ_INVALID_ARG, "contexts of one batch must share a device");
        if (!ctxs[i]->ref || !ctxs[i]->d_walk || ctxs[i]->nwalk == 0)
            return fail(lead, MRQ_NOT_LOADED, "context %d has no initialised walkers", i);
        for (int j = 0; j < i; j++)
            if (ctxs[j] == ctxs[i]) return fail(lead, MRQ_INVALID_ARG, "context %d appears twice", i);
    }
    return 0;
}

// the batch's systems of determinant width W: device tables in the lead context, walker arrays
// from `walkers` (the contexts' own, or the tuner's scratch copies)
// occupancy class of a system in a batch launch: the walk blocks per SM (1-4) its own shared
// memory allows; a batch launches each class separately, so that small systems are not held to the
// occupancy of the largest one
static int batch_class(const mrq_ctx* lead, const mrq_ctx* c, int nw) {
    if (c->W != 1) return 2;
    const long long per = (long long)cta_smem_bytes(std::min(nw, c->max_nw), c->hsys.cand_cap, c->hsys.gstride) +
                          lead->smem_rsv;
    const long long b = per > 0 ? (long long)lead->smem_sm / per : 1;
    return (int)std::max(1LL, std::min(4LL, b));
}

// the systems of one batch launch: width W, warps per walker nw_eff (the requested nw, at most
// what each system's candidate lists allow) and occupancy class cls (0: every class)
static int batch_tables(mrq_ctx* const* ctxs, int n, int W, Walker* const* walkers, WalkSet& ws, int& cap,
                        int& gstride, int cls = 0, int nw = MRQ_MAXNW, int nw_eff = 0) {
    mrq_ctx* ctx = ctxs[0];
    if (n > ctx->bcap) {
        dfree(ctx->d_bsys);
        dfree(ctx->d_bwptr);
        dfree(ctx->d_boff);
        CK(cudaMalloc(&ctx->d_bsys, sizeof(SysDev) * n));
        CK(cudaMalloc(&ctx->d_bwptr, sizeof(Walker*) * n));
        CK(cudaMalloc(&ctx->d_boff, sizeof(long long) * (n + 1)));
        ctx->bcap = n;
    }
    std::vector<SysDev> sys;
    std::vector<Walker*> wp;
    std::vector<long long> off(1, 0);
    cap = 1;
    for (int i = 0; i < n; i++) {
        if (ctxs[i]->W != W) continue;
        if (nw_eff > 0 && std::min(nw, ctxs[i]->max_nw) != nw_eff) continue;
        if (cls > 0 && batch_class(ctx, ctxs[i], nw) != cls) continue;
        sys.push_back(ctxs[i]->hsys);
        wp.push_back(walkers[i]);
        off.push_back(off.back() + ctxs[i]->nwalk);
        cap = std::max(cap, ctxs[i]->hsys.cand_cap);
    }
    ws = WalkSet{ctx->d_bsys, ctx->d_bwptr, ctx->d_boff, (int)sys.size(), off.back()};
    for (size_t k = 0; k + 1 < off.size(); k++) ws.max_seg = std::max(ws.max_seg, off[k + 1] - off[k]);
    gstride = 0;
    for (const SysDev& sd : sys) gstride = std::max(gstride, sd.gstride);
    if (sys.empty()) return 0;
    const int k = (int)sys.size();
    CK(cudaMemcpy(ctx->d_bsys, sys.data(), sizeof(SysDev) * k, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_bwptr, wp.data(), sizeof(Walker*) * k, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_boff, off.data(), sizeof(long long) * (k + 1), cudaMemcpyHostToDevice));
    return 0;
}

// n_steps steps of one width's walk set: launches of `spl` steps (the reporting interval), each
// one sort + one walk, replayed from a CUDA graph when the lead context asks for it
static int batch_run(mrq_ctx* ctx, int W, const WalkSet& ws, int cap, int gstride, int64_t n_steps, int wpb,
                     int64_t spl, int accumulate, bool graph, int slot = -1) {
    if (slot < 0) slot = W - 1;
    WalkLaunch L;
    L.wpb = wpb;
    L.accumulate = accumulate;
    if (spl <= 0 || spl > n_steps) spl = n_steps;
    const int64_t nfull = n_steps / spl, rem = n_steps % spl;
    if (graph && nfull > 0) {
        if (int r = walk_sort_prepare(ctx, ws.nslots, ws.max_seg)) return r;
        if (int r = walk_attr_prepare(ctx, W, cta_smem_bytes(std::min(wpb, MRQ_MAXNW), cap, gstride),
                                      32 * std::min(wpb, MRQ_MAXNW)))
            return r;
        mrq_ctx::GraphKey key;
        key.sys = ws.systems;
        key.wptr = ws.walkers;
        key.off = ws.offsets;
        key.keys = ctx->d_sort_keys;
        key.nslots = ws.nslots;
        key.k = ws.nsys;
        key.wpb = wpb;
        key.spl = (int)spl;
        key.cap = cap;
        key.gstride = gstride;
        cudaGraphExec_t& ex = ctx->gexec[slot];
        if (!ex || !(ctx->gkey[slot] == key)) {
            if (ex) CK(cudaGraphExecDestroy(ex));
            ex = nullptr;
            CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
            L.captured = true;
            const int r = launch_walk(ctx, W, ws, (int)spl, cap, gstride, L);
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
            if (r || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return r ? r : fail(ctx, MRQ_CUDA_ERROR, "stream capture: %s", cudaGetErrorString(e));
            }
            const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) {
                ex = nullptr;
                return fail(ctx, MRQ_CUDA_ERROR, "cudaGraphInstantiate: %s", cudaGetErrorString(ei));
            }
            ctx->gkey[slot] = key;
        }
        for (int64_t i = 0; i < nfull; i++) CK(cudaGraphLaunch(ex, ctx->stream));
        ctx->graph_replays += nfull;
        L.captured = false;
    } else {
        for (int64_t i = 0; i < nfull; i++)
            if (int r = launch_walk(ctx, W, ws, (int)spl, cap, gstride, L)) return r;
    }
    if (rem > 0)
        if (int r = launch_walk(ctx, W, ws, (int)rem, cap, gstride, L)) return r;
    return 0;
}

int mrq_batch_advance(mrq_ctx* const* ctxs, int n, int64_t n_steps) {
    if (int r = batch_check(ctxs, n)) return r;
    mrq_ctx* lead = ctxs[0];
    if (n_steps <= 0) return 0;
    lead->err[0] = 0;
    cudaError_t e0 = cudaSetDevice(lead->device);
    if (e0 != cudaSuccess) return fail(lead, MRQ_CUDA_ERROR, "cudaSetDevice: %s", cudaGetErrorString(e0));
    mrq_ctx* ctx = lead;   // for CK
    for (int i = 0; i < n; i++) CK(cudaStreamSynchronize(ctxs[i]->stream));
    std::vector<Walker*> own(n);
    for (int i = 0; i < n; i++) own[i] = ctxs[i]->d_walk;
    // one launch sequence per determinant width, warps per walker and occupancy class
    for (int slot = 0; slot < mrq_ctx::NSLOT; slot++) {
        const int W = 1 + slot / 16, nw_eff = MRQ_MAXNW >> ((slot / 4) % 4), cls = 4 - slot % 4;
        int nw = lead->wpb;
        if (nw <= 0)
            for (int i = 0; i < n; i++)
                if (ctxs[i]->W == W) nw = std::max(nw, auto_warps(ctxs[i]->hsys));
        WalkSet ws;
        int cap = 1;
        int gstride = 0;
        if (int r = batch_tables(ctxs, n, W, own.data(), ws, cap, gstride, cls, nw, nw_eff)) return r;
        if (ws.nsys == 0) continue;
        const size_t q = (size_t)ctx->launches * 2;
        while (ctx->evs.size() < q + 2) {
            cudaEvent_t ev;
            CK(cudaEventCreate(&ev));
            ctx->evs.push_back(ev);
        }
        CK(cudaEventRecord(ctx->evs[q], ctx->stream));
        if (int r = batch_run(ctx, W, ws, cap, gstride, n_steps, nw_eff, lead->spl, 1, lead->use_graph != 0, slot))
            return r;
        CK(cudaEventRecord(ctx->evs[q + 1], ctx->stream));
        ctx->launches++;
        if (int r_ = sync_stream(ctx)) return r_;   // the tables are reused by the next launch
    }
    for (int i = 0; i < n; i++) ctxs[i]->total_steps += n_steps * ctxs[i]->nwalk;
    return 0;
}

int mrq_set_launch(mrq_ctx* ctx, int warps_per_walker, int steps_per_launch, int use_graph) {
    if (!ctx) return MRQ_INVALID_ARG;
    if (warps_per_walker != 0 && warps_per_walker != 1 && warps_per_walker != 2 && warps_per_walker != 4 &&
        warps_per_walker != 8)
        return fail(ctx, MRQ_INVALID_ARG, "warps_per_walker must be 0 (automatic), 1, 2, 4 or 8");
    if (steps_per_launch < 0) return fail(ctx, MRQ_INVALID_ARG, "steps_per_launch must be >= 0");
    ctx->wpb = warps_per_walker;
    ctx->spl = steps_per_launch;
    ctx->use_graph = use_graph != 0;
    return 0;
}

int mrq_tune_batch(mrq_ctx* const* ctxs, int n, int64_t trial_steps, mrq_tune_result* out) {
    if (int r = batch_check(ctxs, n)) return r;
    mrq_ctx* ctx = ctxs[0];
    if (trial_steps < 1 || trial_steps > 1024) return fail(ctx, MRQ_INVALID_ARG, "trial_steps must be in [1, 1024]");
    ctx->err[0] = 0;
    CK(cudaSetDevice(ctx->device));
    for (int i = 0; i < n; i++) CK(cudaStreamSynchronize(ctxs[i]->stream));
    // scratch copies of every system's walkers: the trials move those, never the real ones
    long long tot = 0;
    for (int i = 0; i < n; i++) tot += ctxs[i]->nwalk;
    if (tot > ctx->tune_cap) {
        dfree(ctx->d_tune);
        CK(cudaMalloc(&ctx->d_tune, sizeof(Walker) * tot));
        ctx->tune_cap = tot;
    }
    std::vector<Walker*> scratch(n);
    {
        long long o = 0;
        for (int i = 0; i < n; i++) {
            scratch[i] = ctx->d_tune + o;
            o += ctxs[i]->nwalk;
        }
    }
    auto restore = [&]() -> int {
        for (int i = 0; i < n; i++)
            CK(cudaMemcpyAsync(scratch[i], ctxs[i]->d_walk, sizeof(Walker) * ctxs[i]->nwalk, cudaMemcpyDeviceToDevice,
                               ctx->stream));
        return 0;
    };
    const int wpbs[3] = {2, 4, 8};
    std::vector<int64_t> spls;
    for (int64_t v : {(int64_t)1, (int64_t)4, (int64_t)16})
        if (v <= trial_steps) spls.push_back(v);
    mrq_tune_result res{};
    double best = 1e300;
    int reps = 3;
    for (int pass = -1; pass < (int)(3 * spls.size()); pass++) {
        const int wpb = pass < 0 ? 8 : wpbs[pass / (int)spls.size()];
        const int64_t spl = pass < 0 ? 1 : spls[pass % spls.size()];
        double ms_best = 1e300;
        for (int rep = 0; rep < (pass < 0 ? 1 : reps); rep++) {
            if (int r = restore()) return r;
            CK(cudaEventRecord(ctx->ev0, ctx->stream));
            for (int slot = 0; slot < mrq_ctx::NSLOT; slot++) {
                const int W = 1 + slot / 16, nw_eff = MRQ_MAXNW >> ((slot / 4) % 4), cls = 4 - slot % 4;
                WalkSet ws;
                int cap = 1;
                int gstride = 0;
                if (int r = batch_tables(ctxs, n, W, scratch.data(), ws, cap, gstride, cls, wpb, nw_eff)) return r;
                if (ws.nsys == 0) continue;
                if (int r = batch_run(ctx, W, ws, cap, gstride, trial_steps, nw_eff, spl, 0, false, slot)) return r;
                if (int r_ = sync_stream(ctx)) return r_;
            }
            CK(cudaEventRecord(ctx->ev1, ctx->stream));
            CK(cudaEventSynchronize(ctx->ev1));
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
            ms_best = std::min(ms_best, (double)ms);
            if (ms > 200.0f) reps = 1;     // long trials: one repetition is precise enough
        }
        if (pass < 0) continue;            // warm-up
        if (res.n_tried < MRQ_TUNE_MAX) {
            res.tried_warps_per_walker[res.n_tried] = wpb;
            res.tried_steps_per_launch[res.n_tried] = (int)spl;
            res.tried_ms[res.n_tried] = ms_best;
            res.n_tried++;
        }
        if (ms_best < best) {
            best = ms_best;
            res.warps_per_walker = wpb;
            res.steps_per_launch = (int)spl;
        }
    }
    for (int i = 0; i < n; i++) {
        ctxs[i]->wpb = res.warps_per_walker;
        ctxs[i]->spl = res.steps_per_launch;
    }
    if (out) *out = res;
    return 0;
}

int mrq_sample_batch(mrq_ctx* const* ctxs, int n, const mrq_sample_params* params, mrq_result* out) {
    if (!ctxs || n <= 0 || !params || !out) return MRQ_INVALID_ARG;
    for (int i = 0; i < n; i++)
        if (params[i].n_steps != params[0].n_steps)
            return fail(ctxs[0], MRQ_INVALID_ARG, "all systems of a batch take the same number of steps");
    for (int i = 0; i < n; i++)
        if (int r = mrq_walkers_init(ctxs[i], &params[i])) return r;
    if (int r = mrq_batch_advance(ctxs, n, params[0].n_steps)) return r;
    int rc = 0;
    for (int i = 0; i < n; i++) {
        int r = mrq_finalize(ctxs[i], &out[i]);
        if (r && !rc) rc = r;
    }
    return rc;
}

int mrq_sample(mrq_ctx* ctx, const mrq_sample_params* p, mrq_result* out) {
    if (int r = mrq_walkers_init(ctx, p)) return r;
    if (!(p->target_sigma > 0.0)) {
        if (int r = mrq_walkers_advance(ctx, p->n_steps)) return r;
        return mrq_finalize(ctx, out);
    }
    const int64_t chunk = p->steps_per_check > 0 ? p->steps_per_check : std::max<int64_t>(1, p->n_steps / 16);
    int64_t done = 0;
    bool fresh = false;
    while (done < p->n_steps) {
        const int64_t k = std::min(chunk, p->n_steps - done);
        if (int r = mrq_walkers_advance(ctx, k)) return r;
        done += k;
        fresh = false;
        if (done <= p->burn_in) continue;
        if (int r = mrq_finalize(ctx, out)) return r;
        fresh = true;
        const double sig = p->method == MRQ_SC_MRCI ? out->e_var_sigma : out->e2_sigma;
        if (sig <= p->target_sigma) break;
    }
    return fresh ? 0 : mrq_finalize(ctx, out);
}

int mrq_read_accumulators(mrq_ctx* ctx, double* accN, double* accU, double* accW, double* accE, int64_t* type_steps) {
    if (!ctx) return MRQ_INVALID_ARG;
    if (!ctx->d_accN) return fail(ctx, MRQ_NOT_LOADED, "no accumulators");
    CK(cudaSetDevice(ctx->device));
    if (int r = sync_stream(ctx)) return r;
    const long long L = ctx->nlab * ctx->G;
    if (accN) CK(cudaMemcpyAsync(accN, ctx->d_accN, sizeof(double) * L, cudaMemcpyDeviceToHost, ctx->stream));
    if (accU) CK(cudaMemcpyAsync(accU, ctx->d_accU, sizeof(double) * L, cudaMemcpyDeviceToHost, ctx->stream));
    if (accW) CK(cudaMemcpyAsync(accW, ctx->d_accW, sizeof(double) * ctx->G, cudaMemcpyDeviceToHost, ctx->stream));
    if (accE) CK(cudaMemcpyAsync(accE, ctx->d_accE, sizeof(double) * ctx->G, cudaMemcpyDeviceToHost, ctx->stream));
    if (type_steps)
        CK(cudaMemcpyAsync(type_steps, ctx->d_types, sizeof(int64_t) * MRQ_NTYPES, cudaMemcpyDeviceToHost, ctx->stream));
    if (int r_ = sync_stream(ctx)) return r_;
    return 0;
}

int mrq_load_accumulators(mrq_ctx* ctx, int32_t n_groups, const double* accN, const double* accU, const double* accW,
                          const double* accE, const double* accA, const double* accB, const int64_t* type_steps,
                          int64_t total_steps) {
    if (!ctx) return MRQ_INVALID_ARG;
    ctx->err[0] = 0;
    if (!ctx->ref) return fail(ctx, MRQ_NOT_LOADED, "no reference loaded");
    if (n_groups <= 0 || n_groups > 64 || !accN || !accU || !accW || !accE || !type_steps || total_steps < 0)
        return fail(ctx, MRQ_INVALID_ARG, "need 1 <= n_groups <= 64, the N, U, W, E sums and the type counts");
    CK(cudaSetDevice(ctx->device));
    if (int r = sync_stream(ctx)) return r;
    DeadlinePause pause_(ctx);
    if (ctx->acc_lab != ctx->nlab || ctx->acc_G != n_groups) {
        dfree(ctx->d_accN);
        dfree(ctx->d_accU);
        dfree(ctx->d_accA);
        dfree(ctx->d_accB);
        dfree(ctx->d_accW);
        dfree(ctx->d_accE);
        dfree(ctx->d_types);
        CK(cudaMalloc(&ctx->d_accN, sizeof(double) * ctx->nlab * n_groups));
        CK(cudaMalloc(&ctx->d_accU, sizeof(double) * ctx->nlab * n_groups));
        CK(cudaMalloc(&ctx->d_accA, sizeof(double) * ctx->nlab * n_groups));
        CK(cudaMalloc(&ctx->d_accB, sizeof(double) * ctx->nlab * n_groups));
        CK(cudaMalloc(&ctx->d_accW, sizeof(double) * n_groups));
        CK(cudaMalloc(&ctx->d_accE, sizeof(double) * n_groups));
        CK(cudaMalloc(&ctx->d_types, sizeof(unsigned long long) * MRQ_NTYPES));
        ctx->acc_lab = ctx->nlab;
        ctx->acc_G = n_groups;
    }
    const long long L = ctx->nlab * n_groups;
    CK(cudaMemcpyAsync(ctx->d_accN, accN, sizeof(double) * L, cudaMemcpyDefault, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_accU, accU, sizeof(double) * L, cudaMemcpyDefault, ctx->stream));
    if (accA) CK(cudaMemcpyAsync(ctx->d_accA, accA, sizeof(double) * L, cudaMemcpyDefault, ctx->stream));
    else CK(cudaMemsetAsync(ctx->d_accA, 0, sizeof(double) * L, ctx->stream));
    if (accB) CK(cudaMemcpyAsync(ctx->d_accB, accB, sizeof(double) * L, cudaMemcpyDefault, ctx->stream));
    else CK(cudaMemsetAsync(ctx->d_accB, 0, sizeof(double) * L, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_accW, accW, sizeof(double) * n_groups, cudaMemcpyDefault, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_accE, accE, sizeof(double) * n_groups, cudaMemcpyDefault, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_types, type_steps, sizeof(int64_t) * MRQ_NTYPES, cudaMemcpyDefault, ctx->stream));
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    ctx->G = n_groups;
    ctx->nwalk = 0;                    // the walkers no longer match the groups: walkers_init first
    ctx->total_steps = total_steps;
    ctx->walk_ms = 0.0;
    ctx->launches = 0;
    if (int r = push_sys(ctx)) return r;
    return sync_stream(ctx);
}

int mrq_read_gradient_sums(mrq_ctx* ctx, double* accA, double* accB) {
    if (!ctx) return MRQ_INVALID_ARG;
    if (!ctx->d_accA) return fail(ctx, MRQ_NOT_LOADED, "no accumulators");
    CK(cudaSetDevice(ctx->device));
    if (int r = sync_stream(ctx)) return r;
    const size_t bytes = sizeof(double) * ctx->nlab * ctx->G;
    if (accA) CK(cudaMemcpyAsync(accA, ctx->d_accA, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    if (accB) CK(cudaMemcpyAsync(accB, ctx->d_accB, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    if (int r_ = sync_stream(ctx)) return r_;
    return 0;
}

int mrq_debug_race_screen(mrq_ctx* ctx, int64_t n, const uint64_t* k53, const double* rate, const double* t_best,
                          uint8_t* pass, double* exact) {
    if (!ctx) return MRQ_INVALID_ARG;
    ctx->err[0] = 0;
    if (n <= 0 || !k53 || !rate || !t_best || !pass || !exact) return fail(ctx, MRQ_INVALID_ARG, "bad arguments");
    for (int64_t i = 0; i < n; i++)
        if (k53[i] >= (1ull << 53)) return fail(ctx, MRQ_INVALID_ARG, "k53[%lld] has more than 53 bits", (long long)i);
    CK(cudaSetDevice(ctx->device));
    unsigned long long* d_k = nullptr;
    double *d_r = nullptr, *d_t = nullptr, *d_e = nullptr;
    unsigned char* d_p = nullptr;
    CK(cudaMalloc(&d_k, sizeof(unsigned long long) * n));
    CK(cudaMalloc(&d_r, sizeof(double) * n));
    CK(cudaMalloc(&d_t, sizeof(double) * n));
    CK(cudaMalloc(&d_e, sizeof(double) * n));
    CK(cudaMalloc(&d_p, n));
    CK(cudaMemcpyAsync(d_k, k53, sizeof(unsigned long long) * n, cudaMemcpyDefault, ctx->stream));
    CK(cudaMemcpyAsync(d_r, rate, sizeof(double) * n, cudaMemcpyDefault, ctx->stream));
    CK(cudaMemcpyAsync(d_t, t_best, sizeof(double) * n, cudaMemcpyDefault, ctx->stream));
    k_race_screen<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(d_k, d_r, d_t, n, d_p, d_e);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(pass, d_p, n, cudaMemcpyDefault, ctx->stream));
    CK(cudaMemcpyAsync(exact, d_e, sizeof(double) * n, cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(d_k);
    cudaFree(d_r);
    cudaFree(d_t);
    cudaFree(d_e);
    cudaFree(d_p);
    return 0;
}

int mrq_set_l2_window(mrq_ctx* ctx, double fraction) {
    if (!ctx) return MRQ_INVALID_ARG;
    if (!(fraction >= 0.0 && fraction <= 1.0)) return fail(ctx, MRQ_INVALID_ARG, "fraction must be in [0, 1]");
    ctx->l2_fraction = fraction;
    return 0;
}

int mrq_set_deadline(mrq_ctx* ctx, double seconds) {
    if (!ctx) return MRQ_INVALID_ARG;
    if (!(seconds >= 0.0)) return fail(ctx, MRQ_INVALID_ARG, "deadline must be >= 0 seconds");
    ctx->deadline_s = seconds;
    return 0;
}

int mrq_debug_set_limits(mrq_ctx* ctx, int max_probe, int cand_cap) {
    if (!ctx) return MRQ_INVALID_ARG;
    if (max_probe < 0 || max_probe > 64 || cand_cap < 0) return fail(ctx, MRQ_INVALID_ARG, "need 0 <= max_probe <= 64, cand_cap >= 0");
    ctx->probe_limit = max_probe;
    ctx->cap_limit = cand_cap;
    if (ctx->ham) {
        CK(cudaSetDevice(ctx->device));
        if (int r = push_sys(ctx)) return r;
    }
    return 0;
}

#ifdef MRQ_PHASE_TIMING
// timing builds only: the walk's per-phase SM cycles since the last call (ten counters)
int mrq_phase_times(unsigned long long* out10) {
    cudaDeviceSynchronize();
    cudaMemcpyFromSymbol(out10, g_phase, sizeof(unsigned long long) * 10);
    unsigned long long z[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    cudaMemcpyToSymbol(g_phase, z, sizeof z);
    return 0;
}
#endif


int mrq_read_walkers(mrq_ctx* ctx, uint64_t* dets, double* psi) {
    if (!ctx) return MRQ_INVALID_ARG;
    if (!ctx->d_walk) return fail(ctx, MRQ_NOT_LOADED, "walkers not initialised");
    CK(cudaSetDevice(ctx->device));
    if (int r = sync_stream(ctx)) return r;
    std::vector<Walker> w(ctx->nwalk);
    CK(cudaMemcpyAsync(w.data(), ctx->d_walk, sizeof(Walker) * ctx->nwalk, cudaMemcpyDeviceToHost, ctx->stream));
    if (int r_ = sync_stream(ctx)) return r_;
    const int W = ctx->W;
    for (long long i = 0; i < ctx->nwalk; i++) {
        if (dets)
            for (int k = 0; k < W; k++) {
                dets[i * 2 * W + k] = w[i].d[0][k];
                dets[i * 2 * W + W + k] = w[i].d[1][k];
            }
        if (psi) psi[i] = w[i].psi;
    }
    return 0;
}

int mrq_set_heat_bath_cutoff(mrq_ctx* ctx, double eps) {
    if (!ctx) return MRQ_INVALID_ARG;
    ctx->err[0] = 0;
    if (!ctx->ham) return fail(ctx, MRQ_NOT_LOADED, "load the Hamiltonian first");
    if (!(eps >= 0.0) || !std::isfinite(eps)) return fail(ctx, MRQ_INVALID_ARG, "the cutoff must be finite and >= 0");
    CK(cudaSetDevice(ctx->device));
    if (int r = sync_stream(ctx)) return r;
    DeadlinePause pause_(ctx);
    ctx->hsys.hb_eps = eps;
    ctx->hsys.hb_on = eps > 0.0 ? 1 : 0;
    if (int r = push_sys(ctx)) return r;
    k_build_tab<<<2432, 256, 0, ctx->stream>>>(ctx->d_sys, ctx->d_tab);
    CK(cudaGetLastError());
    return sync_stream(ctx);
}

int mrq_read_hamiltonian(mrq_ctx* ctx, double* h1, double* eri) {
    if (!ctx) return MRQ_INVALID_ARG;
    ctx->err[0] = 0;
    if (!ctx->ham) return fail(ctx, MRQ_NOT_LOADED, "no Hamiltonian loaded");
    CK(cudaSetDevice(ctx->device));
    if (int r = sync_stream(ctx)) return r;
    if (h1) CK(cudaMemcpyAsync(h1, ctx->d_h1, sizeof(double) * ctx->n * ctx->n, cudaMemcpyDefault, ctx->stream));
    if (eri) CK(cudaMemcpyAsync(eri, ctx->d_eri, sizeof(double) * ctx->neri, cudaMemcpyDefault, ctx->stream));
    return sync_stream(ctx);
}

}  // extern "C"

int mrq_internal_ham(mrq_ctx* ctx, MrqHamView* out) {
    if (!ctx->ham) return fail(ctx, MRQ_NOT_LOADED, "load the Hamiltonian first");
    ctx->err[0] = 0;
    *out = MrqHamView{ctx->device, ctx->stream, ctx->n, ctx->nc, ctx->na, ctx->nv, ctx->nalpha, ctx->nbeta, ctx->W,
                      ctx->d_h1, ctx->d_eri, ctx->neri, ctx->e_nuc};
    return 0;
}

int mrq_internal_fail(mrq_ctx* ctx, int code, const char* fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof ctx->err, fmt, ap);
        va_end(ap);
    }
    return code;
}

int mrq_internal_sync(mrq_ctx* ctx) { return sync_stream(ctx); }

