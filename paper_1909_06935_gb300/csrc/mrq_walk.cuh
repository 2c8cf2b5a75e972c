// The walk step as one thread block per walker (included by mrq.cu after mrq_cas.cuh).
//
// A walker's local evaluation (Eq. 5, Eq. 16, the reach-back overlaps of Eq. 6-7) is split into
// work units that the block's warps take in a fixed interleaved order (warp w: units w, w + NW,
// ...), so every sum is formed in the same order on every run: the step is deterministic.
//
//  * CAS walkers: the neighbours inside the CAS (spin-resolved blocks of active singles and
//    doubles), then every pair (X_a, Y_a) of active electrons removed / active holes filled.  A
//    pair owns the groups (r, spins of the core holes X_c and virtual electrons Y_v) of mrq_cas.cuh,
//    whose neighbours share one reach-back candidate list; large pairs are cut into chunks of
//    neighbours.  The unit plan depends only on the system (all CAS determinants have the same
//    active electron counts), so it is computed on the host at load.
//  * FOIS walkers: chunks of the class-block enumeration of build_lists, reach-back per lane.
//
// Within a unit, rounds of up to 32 neighbours run one neighbour per lane; a round with fewer
// neighbours splits each neighbour's candidate list over f lanes (f a power of two) and reduces
// the f partial sums with shuffles, so short groups keep the lanes busy.
//
// The per-neighbour arithmetic is kept to a few FP64 operations: t = H_nm psi_s(m) is summed as
// |t| and t, and 1/psi_s(n) is applied once per walker (S = |1/psi_n| sum |t|, E_L = H_nn +
// (1/psi_n) sum t); the race screens candidates in FP32 (no logarithm: 1 - u against
// -expm1(-Gamma t_best)) and takes the exact FP64 clock only where a candidate can win.

#ifndef MRQ_MAXNW
#define MRQ_MAXNW 8           // warps per walker block (at most)
#endif
#define MRQ_VW 8              // virtual warps: the fixed partition of a walker's units (MRQ_MAXNW <= MRQ_VW)
#define MRQ_CAS_CH 128        // neighbours per unit inside the CAS
#define MRQ_FOIS_CH 128       // neighbours per unit of a FOIS walker
#define MRQ_UNIT_NB 1024      // neighbours per unit of an (X_a, Y_a) pair (pairs are cut into chunks)
// The walk kernel is compiled for 2, 3 and 4 resident blocks of MRQ_MAXNW warps per SM (128, 80
// and 64 registers); the runtime takes the most blocks the launch's shared memory allows.  More
// resident warps hide more of the gathers' latency: at 56 orbitals (45 KB per block) four blocks
// beat three and three beat two (224, 243 and 263 ms per step); five blocks at 48 registers spill
// too much (268 ms).

// the walker block's shared state (dynamic shared memory starts with it)
struct CasWalker {
    unsigned long long AOn, AEn, keyn;
    int cntO, cntE;
    double phin, c0, inv_psin;
    float inv_psin_f;
};

struct CtaSh {
    WarpSh L;                       // the walker's system (L.sys) and occupied / empty lists
    double wsum[3][MRQ_VW];         // per virtual warp sum |t|, sum t, sum t_D
    double wbt[MRQ_MAXNW];          // per-warp best clock, its psi_s and excitation
    double wbpsi[MRQ_MAXNW];
    unsigned wbexc[MRQ_MAXNW];
    unsigned long long ctr[4];      // debug counters: gathers, probes, candidates, terms
    double hnn, hdnn;
    long long nbase_fois;
    int units;
    int pad_;
    // per-thread race state (best exact clock, its psi_s, FP32 image and excitation): kept in shared
    // memory rather than registers, since it changes only when a candidate beats the lane's best
    double rbt[MRQ_MAXNW * 32];
    double rbpsi[MRQ_MAXNW * 32];
    float rbtf[MRQ_MAXNW * 32];
    unsigned rbexc[MRQ_MAXNW * 32];
    // the walker's determinant and CAS constants, read by the work units from shared memory (the
    // same for every thread; registers stay free for the neighbour loops)
    CasWalker cw;
    unsigned long long nsh[4];
};

__device__ __forceinline__ CtaSh& cta_sh() {
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    return *reinterpret_cast<CtaSh*>(smem_dyn);
}

__host__ __device__ __forceinline__ size_t cta_list_bytes(int cap) {
    return ((size_t)cap * sizeof(double) + (size_t)cap * sizeof(unsigned) + 15) / 16 * 16;
}
__host__ __device__ __forceinline__ size_t cta_smem_bytes(int nw, int cap, int gstride) {
    return (sizeof(CtaSh) + 15) / 16 * 16 + ((size_t)gstride * sizeof(double) + 15) / 16 * 16 +
           (size_t)nw * cta_list_bytes(cap);
}

#ifdef MRQ_PHASE_TIMING
// Phase clock of a timing build (compiled with -DMRQ_PHASE_TIMING only): per-warp SM cycles spent
// in 0 set-up, 1 CAS-internal units, 2 pair-unit overhead, 3 candidate lists, 4 neighbour decode
// and H_nm, 5 reach-back sums, 6 rates / labels / race, 7 FOIS units, 8 block reductions.
__device__ unsigned long long g_phase[10];
struct PhCtr : NoCtr {
    long long t = 0;
    long long acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    __device__ __forceinline__ void mark(int k) {
        const long long u = clock64();
        if (t) acc[k] += u - t;
        t = u;
    }
};
#endif

// per-lane running sums of a walker's step (scaled by 1/psi_s(n) once at the end); the lane's race
// state is in shared memory (CtaSh::rbt ...)
struct LaneAcc2 {
    double sA, sT, sD;     // sum |t|, sum t, sum t_D   (t = H_nm psi_s(m), t_D = (H_D)_nm psi_s(m))
};

__device__ __forceinline__ void acc2_init(LaneAcc2& a) {
    a.sA = a.sT = a.sD = 0.0;
    CtaSh& cs = cta_sh();
    cs.rbt[threadIdx.x] = INFINITY;
    cs.rbtf[threadIdx.x] = INFINITY;
    cs.rbexc[threadIdx.x] = 0xFFFFFFFFu;
    cs.rbpsi[threadIdx.x] = 0.0;
}

// the exact FP64 clock, kept out of the hot loop's code (few candidates pass the screen)
__device__ __noinline__ double race_clock_cold(unsigned long long k53, double g) { return race_clock_f64(k53, g); }

// one neighbour m: sums and the race (Sec. II B first-reaction form).  t = H_nm psi_s(m).
template <int MODE>
__device__ __forceinline__ void lane_post2(const SysDev& S, LaneAcc2& a, double t, double tD, double psim,
                                           double inv_psin, float inv_psin_f, unsigned exc, unsigned step,
                                           unsigned wid) {
    a.sA += fabs(t);
    a.sT += t;
    a.sD += tD;
    if (MODE == MODE_STEP) {
        if ((__double_as_longlong(t) << 1) != 0) {          // t != 0, without an FP64 compare
            const unsigned long long k53 = race_bits(S.seed, exc, step, wid);
            CtaSh& cs = cta_sh();
            const int me = threadIdx.x;
            if (race_may_win(k53, abs_f32_of(t) * inv_psin_f, cs.rbtf[me])) {
                const double g = fabs(t * inv_psin);
                if (g > 0.0) {
                    const double tc = race_clock_cold(k53, g);
                    const double bt = cs.rbt[me];
                    if (tc < bt || (tc == bt && exc < cs.rbexc[me])) {
                        cs.rbt[me] = tc;
                        cs.rbtf[me] = (float)tc;
                        cs.rbexc[me] = exc;
                        cs.rbpsi[me] = psim;
                    }
                }
            }
        }
    }
}

__device__ __forceinline__ void write_rec(mrq_neighbour* rec, const unsigned long long* m, int W, double hnm,
                                          double hd, double om, double psim, double gamma, unsigned exc) {
#pragma unroll
    for (int w = 0; w < 4; w++) rec->det[w] = 0;
    for (int w = 0; w < W; w++) {
        rec->det[w] = m[w];
        rec->det[W + w] = m[2 + w];
    }
    rec->h = hnm;
    rec->hd = hd;
    rec->o = om;
    rec->psi = psim;
    rec->gamma = gamma;
    rec->exc = exc;
    rec->pad = 0;
}

template <int W>
__device__ __forceinline__ void det_words(const unsigned long long (&m)[2][W], unsigned long long* out4) {
    for (int w = 0; w < 2; w++) out4[w] = out4[2 + w] = 0;
#pragma unroll
    for (int w = 0; w < W; w++) {
        out4[w] = m[0][w];
        out4[2 + w] = m[1][w];
    }
}

__device__ __forceinline__ unsigned exc_code(int r1, int r2, int a1, int a2) {
    return (unsigned)r1 | ((unsigned)r2 << 8) | ((unsigned)a1 << 16) | ((unsigned)a2 << 24);
}

// ------------------------------------------------------------------ per-walker constants (CAS)


// spin-resolved candidate blocks: R' (ne electrons of m's active occupation) and A' (nf holes),
// alpha(R') - alpha(A') = dsp; block b takes alpha(R') = ib[b]; its index is decoded by multiplying
// with precomputed reciprocals (mixed radix nRb x nAa x nAb, fastest last)
struct CandPlan {
    unsigned long long oa, ob, ea, eb;   // m's active electrons / holes by spin (combined bit positions)
    int coa, cob, cea, ceb;
    int nblk;
    int ib[3];
    int start[4];
    unsigned rAb[3], rAa[3], rRb[3];     // the radices and their magic32 reciprocals
    unsigned mAb[3], mAa[3], mRb[3];
};

__device__ __forceinline__ void cand_plan(CandPlan& P, unsigned long long AOm, unsigned long long AEm, int ne, int nf,
                                          int dsp) {
    P.oa = AOm & 0xFFFFFFFFull;
    P.ob = AOm & 0xFFFFFFFF00000000ull;
    P.ea = AEm & 0xFFFFFFFFull;
    P.eb = AEm & 0xFFFFFFFF00000000ull;
    P.coa = __popcll(P.oa);
    P.cob = __popcll(P.ob);
    P.cea = __popcll(P.ea);
    P.ceb = __popcll(P.eb);
    P.nblk = 0;
    P.start[0] = 0;
    for (int i = 0; i <= ne; i++) {
        const int j = i - dsp;
        if (j < 0 || j > nf) continue;
        if (i > P.coa || ne - i > P.cob || j > P.cea || nf - j > P.ceb) continue;
        const int nRa = nsub(P.coa, i), nRb = nsub(P.cob, ne - i), nAa = nsub(P.cea, j), nAb = nsub(P.ceb, nf - j);
        const int sz = nRa * nRb * nAa * nAb;
        if (sz == 0) continue;
        const int b = P.nblk;
        P.ib[b] = i;
        P.rAb[b] = (unsigned)nAb;
        P.rAa[b] = (unsigned)nAa;
        P.rRb[b] = (unsigned)nRb;
        P.mAb[b] = magic32((unsigned)nAb);
        P.mAa[b] = magic32((unsigned)nAa);
        P.mRb[b] = magic32((unsigned)nRb);
        P.start[b + 1] = P.start[b] + sz;
        P.nblk++;
    }
}

__device__ __forceinline__ void cand_decode(const SysDev& S, const CandPlan& P, int ne, int nf, int dsp, int t,
                                            unsigned long long& Rb, unsigned long long& Ab) {
    int b = 0;
    while (b + 1 < P.nblk && t >= P.start[b + 1]) b++;
    unsigned x = (unsigned)(t - P.start[b]);
    const int i = P.ib[b], j = i - dsp;
    unsigned q = div_m(x, P.mAb[b]);
    const int tAb = (int)(x - q * P.rAb[b]);
    x = q;
    q = div_m(x, P.mAa[b]);
    const int tAa = (int)(x - q * P.rAa[b]);
    x = q;
    q = div_m(x, P.mRb[b]);
    const int tRb = (int)(x - q * P.rRb[b]);
    const int tRa = (int)q;
    Rb = subset_bits(S.colex, P.oa, P.coa, i, tRa) | subset_bits(S.colex, P.ob, P.cob, ne - i, tRb);
    Ab = subset_bits(S.colex, P.ea, P.cea, j, tAa) | subset_bits(S.colex, P.eb, P.ceb, nf - j, tAb);
}

// build the candidate list of group (c, v, sc, sv) of active remnant (AOm, AEm): singles [0, n1) as
// codes, doubles [n1, count) as (signed weight, table base); the candidate k = n is left out.  Kept
// out of line: it runs once per group, and its registers and code then stay out of the neighbour
// loop that follows (1.8 % faster at 56 orbitals)
template <int W, class C>
__device__ __noinline__ int build_group_list(const SysDev& S, const CasWalker& cw,
                                                const unsigned long long (&mref)[2][W], unsigned long long AOm,
                                                unsigned long long AEm, int c, int v, int sc, int sv, int rxc0,
                                                int rxc1, int ryv0, int ryv1, int par_ref, double* cphi,
                                                unsigned* ccode, int& n1, int lane, C& ctr) {
    const unsigned lt = (1u << lane) - 1u;
    int count = 0;
    n1 = 0;
    for (int rr = 1; rr <= 2; rr++) {
        if (rr == 2) n1 = count;
        if (rr == 1 && (c > 1 || v > 1)) continue;
        const int ne = rr - v, nf = rr - c;
        if (ne < 0 || nf < 0) continue;
        const int dsp = sc - sv;                  // alpha(R') - alpha(A') = alpha(X_c) - alpha(Y_v)
        CandPlan P;
        cand_plan(P, AOm, AEm, ne, nf, dsp);
        const int tot = P.start[P.nblk];
        for (int base = 0; base < tot; base += 32) {
            const int t = base + lane;
            bool valid = t < tot;
            unsigned long long Rb = 0, Ab = 0;
            double phi = 0.0;
            if (valid) {
                cand_decode(S, P, ne, nf, dsp, t, Rb, Ab);
                const unsigned long long kact = (AOm & ~Rb) | Ab;
                const unsigned long long key = hash_key(S, (unsigned)kact, (unsigned)(kact >> 32));
                ctr.cand();
                if (key == cw.keyn) valid = false;
                else {
                    phi = hash_lookup(S, key, ctr);
                    valid = (__double_as_longlong(phi) << 1) != 0;      // phi != 0 without an FP64 compare
                }
            }
            const unsigned vm = __ballot_sync(0xffffffffu, valid);
            if (valid) {
                const int pos = count + __popc(vm & lt);
                if (pos < S.cand_cap) {
                    if (rr == 1) {
                        cphi[pos] = phi;
                        ccode[pos] = pack_cand(Rb, Ab, rr);
                    } else {
                        double w;
                        unsigned bp;
                        dbl_entry<W>(S, mref, c, v, rxc0, rxc1, ryv0, ryv1, par_ref, Rb, Ab, phi, w, bp);
                        cphi[pos] = w;
                        ccode[pos] = bp;
                    }
                }
            }
            count += __popc(vm);
        }
    }
    if (count > S.cand_cap) {
        if (lane == 0) atomicOr(S.err, MRQ_ERR_CAP);
        count = S.cand_cap;
        n1 = min(n1, count);
    }
    __syncwarp();
    return count;
}

// lanes per neighbour in a round of nr neighbours
__device__ __forceinline__ int split_of(int nr) {
    return nr > 16 ? 1 : (nr > 8 ? 2 : (nr > 4 ? 4 : (nr > 2 ? 8 : (nr > 1 ? 16 : 32))));
}

// <m|H|n> of a double n -> m (removed r1 < r2 core/active, added a1 < a2 active/virtual) from the
// physicists' tables: <r1 r2||a1 a2> (same spin) or <r1 r2|a1 a2> (opposite), one gather
template <int W, class C>
__device__ __forceinline__ double double_elem_tab(const SysDev& S, const unsigned long long (&d)[2][W], int r1, int r2,
                                                  int a1, int a2, C& ctr) {
    const int n = S.n;
    const int s_r1 = r1 >= n, s_r2 = r2 >= n;
    const int pr1 = r1 - s_r1 * n, pr2 = r2 - s_r2 * n, pa1 = a1 - (a1 >= n) * n, pa2 = a2 - (a2 >= n) * n;
    int c1 = popc_sel<W>(d, s_r1, min(pr1, pa1), max(pr1, pa1));
    int c2;
    if (s_r2 == s_r1) {
        unsigned long long t[W];
#pragma unroll
        for (int w = 0; w < W; w++) t[w] = s_r1 ? d[1][w] : d[0][w];
        flip<W>(t, pr1);
        flip<W>(t, pa1);
        c2 = popc_between<W>(t, min(pr2, pa2), max(pr2, pa2));
    } else {
        c2 = popc_sel<W>(d, s_r2, min(pr2, pa2), max(pr2, pa2));
    }
    const unsigned sv = (unsigned)S.nav, sq = sv * sv, sp = sq * (unsigned)S.nca;
    const unsigned idx = (s_r1 == s_r2 ? S.tab_half : 0u) + (unsigned)pr1 * sp + (unsigned)pr2 * sq +
                         (unsigned)(pa1 - S.nc) * sv + (unsigned)(pa2 - S.nc);
    ctr.g();
    return neg_if(__ldg(S.tab + idx), c1 + c2);
}

// ------------------------------------------------------------------ CAS units

// neighbours of pair (X_a, Y_a) in the flat order of its groups; returns the total
__device__ __forceinline__ int pair_total(const SysDev& S, int ka, int kb, int d) {
    int tot = 0;
    for (int r = max(1, max(ka, kb)); r <= 2; r++) {
        const int c = r - ka, v = r - kb;
        if (c == 0 && v == 0) continue;
        for (int sc = 0; sc <= c; sc++) {
            const int sv = sc - d;
            if (sv < 0 || sv > v) continue;
            tot += shape_count(S.nc, c, sc) * shape_count(S.nv, v, sv);
        }
    }
    return tot;
}

// neighbours of one CAS unit (for the debug records' offsets)
__device__ __forceinline__ int cas_unit_count(const SysDev& S, const CasWalker& cw, int u) {
    if (u < S.cas_units) return min(MRQ_CAS_CH, S.cas_nb - u * MRQ_CAS_CH);
    int k = 0;
    while (k < 7 && u >= S.unit_off[k + 1]) k++;
    const int ka = k / 3, kb = k % 3, nch = S.nch[k];
    const int loc = u - S.unit_off[k];
    const int pair = loc / nch, ch = loc - pair * nch;
    const int nYa = nsub(cw.cntE, kb);
    const int xa = pair / nYa, ya = pair - xa * nYa;
    const unsigned long long Xb = subset_bits(S.colex, cw.AOn, cw.cntO, ka, xa);
    const unsigned long long Yb = subset_bits(S.colex, cw.AEn, cw.cntE, kb, ya);
    const int d = __popcll(Yb & 0xFFFFFFFFull) - __popcll(Xb & 0xFFFFFFFFull);
    const int tot = pair_total(S, ka, kb, d);
    const int lo = (int)((long long)ch * tot / nch), hi = (int)((long long)(ch + 1) * tot / nch);
    return hi - lo;
}

// neighbours inside the CAS: spin-resolved blocks (alpha singles, beta singles, alpha-alpha,
// beta-beta, alpha-beta doubles) of the walker's active electrons / holes
template <int W, int MODE, class C>
__device__ __noinline__ LaneAcc2 cas_internal_unit(const SysDev& S, const CasWalker& cw, const unsigned long long (&n)[2][W], int u,
                                  LaneAcc2 acc, unsigned step, unsigned wid, int lane, mrq_neighbour* nbout,
                                  long long nbase, long long max_nb, C& ctr) {
    const unsigned long long oa = cw.AOn & 0xFFFFFFFFull, ob = cw.AOn & ~0xFFFFFFFFull;
    const unsigned long long ea = cw.AEn & 0xFFFFFFFFull, eb = cw.AEn & ~0xFFFFFFFFull;
    const int coa = __popcll(oa), cob = __popcll(ob), cea = __popcll(ea), ceb = __popcll(eb);
    const int b0 = coa * cea, b1 = b0 + cob * ceb, b2 = b1 + nsub(coa, 2) * nsub(cea, 2),
              b3 = b2 + nsub(cob, 2) * nsub(ceb, 2), b4 = b3 + coa * cea * cob * ceb;
    const int i0 = u * MRQ_CAS_CH, i1 = min(b4, i0 + MRQ_CAS_CH);
    for (int idx = i0 + lane; idx < i1; idx += 32) {
        unsigned long long Xb, Yb;
        int r;
        if (idx < b0) {
            r = 1;
            Xb = subset_bits(S.colex, oa, coa, 1, idx / cea);
            Yb = subset_bits(S.colex, ea, cea, 1, idx % cea);
        } else if (idx < b1) {
            const int x = idx - b0;
            r = 1;
            Xb = subset_bits(S.colex, ob, cob, 1, x / ceb);
            Yb = subset_bits(S.colex, eb, ceb, 1, x % ceb);
        } else if (idx < b2) {
            const int x = idx - b1, ny = nsub(cea, 2);
            r = 2;
            Xb = subset_bits(S.colex, oa, coa, 2, x / ny);
            Yb = subset_bits(S.colex, ea, cea, 2, x % ny);
        } else if (idx < b3) {
            const int x = idx - b2, ny = nsub(ceb, 2);
            r = 2;
            Xb = subset_bits(S.colex, ob, cob, 2, x / ny);
            Yb = subset_bits(S.colex, eb, ceb, 2, x % ny);
        } else {
            int x = idx - b3;
            r = 2;
            const int yb = x % ceb;
            x /= ceb;
            const int xb = x % cob;
            x /= cob;
            const int ya = x % cea, xa = x / cea;
            Xb = subset_bits(S.colex, oa, coa, 1, xa) | subset_bits(S.colex, ob, cob, 1, xb);
            Yb = subset_bits(S.colex, ea, cea, 1, ya) | subset_bits(S.colex, eb, ceb, 1, yb);
        }
        int rem[2], add[2];
        act_list(S, Xb, rem);
        act_list(S, Yb, add);
        unsigned long long m[2][W];
#pragma unroll
        for (int sg = 0; sg < 2; sg++)
#pragma unroll
            for (int w = 0; w < W; w++) m[sg][w] = n[sg][w];
        apply_exc<W>(m, S, rem, add, r);
        const double hnm = r == 1 ? single_elem<W>(S, n, rem[0], add[0], ctr)
                                  : double_elem_tab<W>(S, n, rem[0], rem[1], add[0], add[1], ctr);
        const unsigned long long km = (cw.AOn & ~Xb) | Yb;
        ctr.cand();
        const double om = hash_lookup(S, hash_key(S, (unsigned)km, (unsigned)(km >> 32)), ctr);
        const unsigned exc = r == 1 ? exc_code(rem[0], rem[0], add[0], add[0]) : exc_code(rem[0], rem[1], add[0], add[1]);
        const double psim = cw.c0 * om;
        const double t = hnm * psim;
        lane_post2<MODE>(S, acc, t, 0.0, psim, cw.inv_psin, cw.inv_psin_f, exc, step, wid);
        if (MODE == MODE_DEBUG && nbout != nullptr && nbase + (idx - i0) < max_nb) {
            unsigned long long w4[4];
            det_words<W>(m, w4);
            write_rec(nbout + nbase + (idx - i0), w4, W, hnm, 0.0, om, psim, fabs(t * cw.inv_psin), exc);
        }
    }
    return acc;
}

// one (X_a, Y_a) pair chunk [lo, hi) of a CAS walker
template <int W, int MODE, class C>
__device__ void cas_pair_unit(const SysDev& S, const CasWalker& cw, const double* __restrict__ gops, double* cphi,
                              unsigned* ccode, const unsigned long long (&n)[2][W], int u, LaneAcc2& acc,
                              unsigned step, unsigned wid, int lane, mrq_neighbour* nbout, long long nbase,
                              long long max_nb, C& ctr) {
    int k = 0;
    while (k < 7 && u >= S.unit_off[k + 1]) k++;
    const int ka = k / 3, kb = k % 3, nch = S.nch[k];
    const int loc = u - S.unit_off[k];
    const int pair = loc / nch, ch = loc - pair * nch;
    const int nYa = nsub(cw.cntE, kb);
    const int xa = pair / nYa, ya = pair - xa * nYa;
    const unsigned long long Xb = subset_bits(S.colex, cw.AOn, cw.cntO, ka, xa);
    const unsigned long long Yb = subset_bits(S.colex, cw.AEn, cw.cntE, kb, ya);
    const int d = __popcll(Yb & 0xFFFFFFFFull) - __popcll(Xb & 0xFFFFFFFFull);
    const int tot = pair_total(S, ka, kb, d);
    const int lo = (int)((long long)ch * tot / nch), hi = (int)((long long)(ch + 1) * tot / nch);
    if (lo >= hi) return;
    const unsigned long long AOm = (cw.AOn & ~Xb) | Yb, AEm = (cw.AEn & ~Yb) | Xb;
    const int xa0 = Xb ? act_so(S, __ffsll(Xb) - 1) : 0;
    const int xa1 = (ka == 2) ? act_so(S, 63 - __clzll(Xb)) : 0;
    const int ya0 = Yb ? act_so(S, __ffsll(Yb) - 1) : 0;
    const int ya1 = (kb == 2) ? act_so(S, 63 - __clzll(Yb)) : 0;
    const int nc = S.nc, nv = S.nv, voff = S.nc + S.na;
    int base = 0;
    ctr.mark(2);
    for (int r = max(1, max(ka, kb)); r <= 2; r++) {
        const int c = r - ka, v = r - kb;
        if (c == 0 && v == 0) continue;
        for (int sc = 0; sc <= c; sc++) {
            const int sv = sc - d;
            if (sv < 0 || sv > v) continue;
            const int ncc = shape_count(nc, c, sc), nvc = shape_count(nv, v, sv);
            const int ni = ncc * nvc;
            const int q0 = max(lo, base) - base, q1 = min(hi, base + ni) - base;
            if (ni > 0 && q0 < q1) {
                // reference neighbour (the group's first) for the candidates' signs
                int rxc0, rxc1, ryv0, ryv1, rrm0, rrm1, rad0, rad1;
                unsigned long long mref[2][W];
                group_neighbour<W>(S, n, nc, nv, voff, c, sc, v, sv, 0, 0, ka, xa0, xa1, kb, ya0, ya1, r, rxc0, rxc1,
                                   ryv0, ryv1, rrm0, rrm1, rad0, rad1, mref);
                const int par_ref = (c >= 1 ? rxc0 - (rxc0 >= S.n ? S.n : 0) : 0) + (c == 2 ? rxc1 - (rxc1 >= S.n ? S.n : 0) : 0);
                int n1;
                // floor(q / nvc) = high word of q * ceil(2^64 / nvc), exact for q < 2^32 (nvc > 1)
                const unsigned long long mvc = ~0ull / (unsigned long long)nvc + 1ull;
                ctr.mark(2);
                const int count = build_group_list<W>(S, cw, mref, AOm, AEm, c, v, sc, sv, rxc0, rxc1, ryv0, ryv1,
                                                      par_ref, cphi, ccode, n1, lane, ctr);
                ctr.mark(3);
                for (int qb = q0; qb < q1; qb += 32) {
                    const int nr = min(32, q1 - qb);
                    const int f = split_of(nr), lf = __ffs(f) - 1;
                    const int qi = lane >> lf, part = lane & (f - 1);
                    const bool valid = qi < nr;
                    const int q = qb + (valid ? qi : 0);
                    int xc0, xc1, yv0, yv1, rm0, rm1, ad0, ad1;
                    unsigned long long m[2][W];
                    const int ic = nvc == 1 ? q : (int)__umul64hi((unsigned long long)q, mvc);     // q / nvc
                    group_neighbour<W>(S, n, nc, nv, voff, c, sc, v, sv, ic, q - ic * nvc, ka, xa0, xa1, kb, ya0,
                                       ya1, r, xc0, xc1, yv0, yv1, rm0, rm1, ad0, ad1, m);
                    unsigned offd, offx;
                    int par;
                    lane_offsets(S, c, v, xc0, xc1, yv0, yv1, offd, offx, par);
                    double hnm = 0.0, a0 = 0.0, a1 = 0.0;
                    ctr.mark(4);
                    if (valid) {
                        if (part == 0) {
                            if (r == 1) {
                                // single n -> m (x = rm0 -> y = ad0): the walker's operator G
                                const int sx = rm0 >= S.n, px = rm0 - sx * S.n, py = ad0 - sx * S.n;
                                hnm = neg_if(gops[(sx * S.nca + px) * S.nav + (py - S.nc)],
                                             sgn_sel<W>(n, sx, px, py) < 0 ? 1 : 0);
                                ctr.g();
                            } else {
                                hnm = double_elem_tab<W>(S, n, rm0, rm1, ad0, ad1, ctr);
                            }
                            a0 = neg_if(hnm * cw.phin, par);        // the k = n term
                        }
                        ctr.mark(4);
                        for (int e = part; e < n1; e += f)
                            a1 = fma(cphi[e], neg_if(sgl_elem_code<W>(S, gops, m, ccode[e], v, yv0, c, xc0, r, rm0,
                                                                       rm1, ad0, ad1, ctr), par), a1);
                        int e = n1 + ((part - n1) & (f - 1));
                        const int st = f;
                        for (; e + 3 * st < count; e += 4 * st) {
                            const unsigned p0 = ccode[e], p1 = ccode[e + st], p2 = ccode[e + 2 * st],
                                           p3 = ccode[e + 3 * st];
                            const double x0 = __ldg(S.tab + (p0 & 0x7FFFFFFFu) + ((p0 & 0x80000000u) ? offx : offd));
                            const double x1 = __ldg(S.tab + (p1 & 0x7FFFFFFFu) + ((p1 & 0x80000000u) ? offx : offd));
                            const double x2 = __ldg(S.tab + (p2 & 0x7FFFFFFFu) + ((p2 & 0x80000000u) ? offx : offd));
                            const double x3 = __ldg(S.tab + (p3 & 0x7FFFFFFFu) + ((p3 & 0x80000000u) ? offx : offd));
                            a0 = fma(cphi[e], x0, a0);
                            a1 = fma(cphi[e + st], x1, a1);
                            a0 = fma(cphi[e + 2 * st], x2, a0);
                            a1 = fma(cphi[e + 3 * st], x3, a1);
                            ctr.g(4);
                        }
                        for (; e < count; e += st) {
                            const unsigned p0 = ccode[e];
                            a0 = fma(cphi[e], __ldg(S.tab + (p0 & 0x7FFFFFFFu) + ((p0 & 0x80000000u) ? offx : offd)), a0);
                            ctr.g();
                        }
                    }
                    double s = a0 + a1;
                    for (int o = f >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                    ctr.mark(5);
                    if (valid && part == 0) {
                        ctr.term(count + 1);
                        const double om = neg_if(s, par);
                        const int h0 = xc0 >= S.n ? nc + (xc0 - S.n) : xc0;
                        const int h1 = xc1 >= S.n ? nc + (xc1 - S.n) : xc1;
                        const int p0 = yv0 >= S.n ? nv + (yv0 - S.n - voff) : yv0 - voff;
                        const int p1 = yv1 >= S.n ? nv + (yv1 - S.n - voff) : yv1 - voff;
                        const long long lm = set_rank(c, h0, h1, 2 * nc) * S.nPs + set_rank(v, p0, p1, 2 * nv);
                        ctr.g();
                        const double psim = __ldg(S.c + lm) * om;
                        const double t = hnm * psim;
                        const unsigned exc = r == 1 ? exc_code(rm0, rm0, ad0, ad0) : exc_code(rm0, rm1, ad0, ad1);
                        lane_post2<MODE>(S, acc, t, 0.0, psim, cw.inv_psin, cw.inv_psin_f, exc, step, wid);
                        if (MODE == MODE_DEBUG && nbout != nullptr) {
                            const long long ri = nbase + (base + q) - lo;
                            if (ri < max_nb) {
                                unsigned long long w4[4];
                                det_words<W>(m, w4);
                                write_rec(nbout + ri, w4, W, hnm, 0.0, om, psim, fabs(t * cw.inv_psin), exc);
                            }
                        }
                    }
                    ctr.mark(6);
                }
                __syncwarp();
            }
            base += ni;
        }
    }
}

// ------------------------------------------------------------------ FOIS units

// neighbours [i0, i1) of the class-block enumeration, reach-back per lane
template <int W, int MODE, class C>
__device__ __noinline__ LaneAcc2 fois_unit(const SysDev& S, const WarpSh& sh, const double* __restrict__ gops,
                          const unsigned long long (&n)[2][W], long long ln,
                          double c0, double inv_psin, float inv_psin_f, unsigned long long self_key, double phi_self,
                          int i0, int i1, LaneAcc2 acc, unsigned step, unsigned wid, int lane, mrq_neighbour* nbout,
                          long long nbase, long long max_nb, C& ctr) {
    for (int idx = i0 + lane; idx < i1; idx += 32) {
        int lo = 0, hi = sh.nb - 1;          // block of idx: last b with bstart[b] <= idx
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sh.bstart[mid] <= idx) lo = mid;
            else hi = mid - 1;
        }
        const unsigned desc = sh.bdesc[lo];
        int kind, r1, r2, a1, a2;
        decode_exc(sh, S.n, desc, idx - sh.bstart[lo], kind, r1, r2, a1, a2);
        unsigned long long m[2][W];
#pragma unroll
        for (int sg = 0; sg < 2; sg++)
#pragma unroll
            for (int w = 0; w < W; w++) m[sg][w] = n[sg][w];
        {
            int s1 = r1 >= S.n, s2 = a1 >= S.n;
            flip_reg<W>(m, s1, r1 - s1 * S.n);
            flip_reg<W>(m, s2, a1 - s2 * S.n);
            if (kind != 0) {
                int s3 = r2 >= S.n, s4 = a2 >= S.n;
                flip_reg<W>(m, s3, r2 - s3 * S.n);
                flip_reg<W>(m, s4, a2 - s4 * S.n);
            }
        }
        double hnm;
        if (kind != 0) hnm = hb_screen(S, double_elem<W>(S, n, r1, r2, a1, a2, ctr));
        else if (gops != nullptr && in_walker_block(S, r1, a1))
            hnm = single_from_walker<W>(S, SglFromWalker{gops, 0, 0, 0, 0, 0}, n, r1, a1, ctr);
        else hnm = single_elem<W>(S, n, r1, a1, ctr);
        int hm, pm;
        const long long lm = det_label<W>(S, m, hm, pm);
        double om, psim;
        if (lm == 0) {
            ctr.cand();
            om = hash_lookup(S, hash_key(S, active_bits<W>(S, m[0]), active_bits<W>(S, m[1])), ctr);
            psim = c0 * om;
        } else {
            om = reach_back<W>(S, m, ctr, self_key, hnm * phi_self,
                               SglFromWalker{gops, kind == 0 ? 1 : 2, r1, r2, a1, a2});
            ctr.g();
            psim = __ldg(S.c + lm) * om;
        }
        const bool same = ln > 0 && active_only(desc);
        const double hd = same ? ((kind == 0) ? hd_single_elem<W>(S, n, r1, a1, ctr) : hnm) : 0.0;
        const unsigned exc = exc_code(r1, r2, a1, a2);
        const double t = hnm * psim;
        lane_post2<MODE>(S, acc, t, hd * psim, psim, inv_psin, inv_psin_f, exc, step, wid);
        if (MODE == MODE_DEBUG && nbout != nullptr && nbase + idx < max_nb) {
            unsigned long long w4[4];
            det_words<W>(m, w4);
            write_rec(nbout + nbase + idx, w4, W, hnm, hd, om, psim, fabs(t * inv_psin), exc);
        }
    }
    return acc;
}

// ------------------------------------------------------------------ one walker step per block

template <class C>
__device__ __forceinline__ void ctr_flush(CtaSh& cs, const C& ctr, int lane) {}
template <>
__device__ __forceinline__ void ctr_flush<Ctr>(CtaSh& cs, const Ctr& ctr, int lane) {
    unsigned long long v[4] = {ctr.gathers, ctr.probes, ctr.cands, ctr.terms};
#pragma unroll
    for (int k = 0; k < 4; k++) {
        unsigned long long x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) atomicAdd(&cs.ctr[k], x);
    }
}

struct StepOut {
    double S, EL, num, hnn, hdnn;
    long long nnb;
    unsigned bexc;
    double bpsi;
};

// The local evaluation of determinant n (psi_s(n) = psin, label ln, (h, p)) by the whole block.
// Returns on every thread; the winner of the race is valid in MODE_STEP.
template <int W, int MODE, class C>
__device__ StepOut block_local(CtaSh& cs, unsigned char* lists, const unsigned long long (&n)[2][W], double psin,
                               long long ln, int h, int p, unsigned step, unsigned wid, mrq_neighbour* nbout,
                               long long max_nb, long long* nb_prefix, C& ctr) {
    const SysDev& S = cs.L.sys;
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double c0 = __ldg(S.c);
    const double inv_psin = psin != 0.0 ? 1.0 / psin : 0.0;
    const float inv_psin_f = abs_f32_of(inv_psin);
    double* gops = reinterpret_cast<double*>(lists);
    unsigned char* wl = lists + ((size_t)S.gstride * sizeof(double) + 15) / 16 * 16 + (size_t)wi * cta_list_bytes(S.cand_cap);
    double* cphi = reinterpret_cast<double*>(wl);
    unsigned* ccode = reinterpret_cast<unsigned*>(cphi + S.cand_cap);
    if (wi == 0) build_lists<W>(S, n, cs.L, ln == 0 ? 0 : h, ln == 0 ? 0 : p, lane);
    CasWalker cw;
    const bool cas = ln == 0 && psin != 0.0;
    int units;
    if (cas) {
        const unsigned ao0 = active_bits<W>(S, n[0]), ao1 = active_bits<W>(S, n[1]);
        const unsigned amask = (S.na >= 32) ? 0xFFFFFFFFu : ((1u << S.na) - 1u);
        cw.AOn = (unsigned long long)ao0 | ((unsigned long long)ao1 << 32);
        cw.AEn = (unsigned long long)(~ao0 & amask) | ((unsigned long long)(~ao1 & amask) << 32);
        cw.keyn = hash_key(S, ao0, ao1);
        cw.cntO = __popcll(cw.AOn);
        cw.cntE = __popcll(cw.AEn);
        cw.c0 = c0;
        cw.phin = psin / c0;
        cw.inv_psin = inv_psin;
        cw.inv_psin_f = inv_psin_f;
        units = S.unit_off[8];
        if (threadIdx.x == 0) cs.cw = cw;
    }
    // the walker's single-excitation operator G_yx(n) = h_yx + sum_{j in n} [(yx|jj) - delta (yj|jx)]
    // for y in core + active, x in active + virtual (not both active), by the whole block: the
    // full-core operator hc, n's active electrons, minus n's core holes, plus its virtual electrons
    if (psin != 0.0) {
        const unsigned ao0 = active_bits<W>(S, n[0]), ao1 = active_bits<W>(S, n[1]);
        const unsigned long long AOn = (unsigned long long)ao0 | ((unsigned long long)ao1 << 32);
        int nh = 0, np = 0, hso[2] = {0, 0}, pso[2] = {0, 0};
        if (!cas) {
#pragma unroll
            for (int sg = 0; sg < 2; sg++) {
                unsigned long long hm = ~(sg ? n[1][0] : n[0][0]) & S.mcore[0];
                while (hm) {
                    const int i = __ffsll(hm) - 1;
                    hm &= hm - 1;
                    if (nh == 0) hso[0] = sg * S.n + i;
                    else hso[1] = sg * S.n + i;
                    nh++;
                }
#pragma unroll
                for (int w = 0; w < W; w++) {
                    unsigned long long pm = (sg ? n[1][w] : n[0][w]) & S.mvirt[w];
                    while (pm) {
                        const int a = 64 * w + __ffsll(pm) - 1;
                        pm &= pm - 1;
                        if (np == 0) pso[0] = sg * S.n + a;
                        else pso[1] = sg * S.n + a;
                        np++;
                    }
                }
            }
        }
        const int blk = S.nca * S.nav;
        for (int t = threadIdx.x; t < 2 * blk; t += blockDim.x) {
            const int sg = t >= blk, rem = t - sg * blk;
            const int y = rem / S.nav, xo = rem - y * S.nav, x = S.nc + xo;
            if (y >= S.nc && xo < S.na) continue;
            ctr.g();
            double v = __ldg(S.hc + y * S.n + x);
            unsigned long long bits = AOn;
            while (bits) {
                const int b = __ffsll(bits) - 1;
                bits &= bits - 1;
                const int j = S.nc + (b & 31);
                v += eri_g(S, y, x, j, j);
                ctr.g();
                if ((b >= 32) == (sg == 1)) {
                    v -= eri_g(S, y, j, j, x);
                    ctr.g();
                }
            }
#pragma unroll
            for (int k = 0; k < 2; k++) {
                if (k < nh) {
                    v -= g_corr(S, sg, x, y, hso[k]);
                    ctr.g(2);
                }
                if (k < np) {
                    v += g_corr(S, sg, x, y, pso[k]);
                    ctr.g(2);
                }
            }
            gops[t] = v;
        }
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int sg = 0; sg < 2; sg++)
#pragma unroll
            for (int w = 0; w < W; w++) cs.nsh[sg * W + w] = n[sg][w];
    }
    const unsigned long long(&nsh)[2][W] = *reinterpret_cast<const unsigned long long(*)[2][W]>(cs.nsh);
    __syncthreads();
    ctr.mark(0);
    const int total_fois = cas ? 0 : cs.L.bstart[cs.L.nb];
    if (!cas) units = (total_fois + MRQ_FOIS_CH - 1) / MRQ_FOIS_CH;
    // neighbour offsets of the units (debug records only)
    if (MODE == MODE_DEBUG && nbout != nullptr && cas) {
        for (int u = threadIdx.x; u < units; u += blockDim.x) nb_prefix[u] = cas_unit_count(S, cw, u);
        __syncthreads();
        if (threadIdx.x == 0) {
            long long run = 0;
            for (int u = 0; u < units; u++) {
                const long long c = nb_prefix[u];
                nb_prefix[u] = run;
                run += c;
            }
        }
        __syncthreads();
    }
    LaneAcc2 acc;
    acc2_init(acc);
    const unsigned long long self_key =
        ln == 0 ? hash_key(S, active_bits<W>(S, n[0]), active_bits<W>(S, n[1])) : MRQ_EMPTY_KEY;
    const double phi_self = ln == 0 ? psin / c0 : 0.0;
    // MRQ_VW virtual warps: virtual warp v owns units v, v + MRQ_VW, ...; warp wi runs virtual warps
    // wi, wi + nw, ... one after the other and stores each one's sums.  The sums (and so S, E_L and
    // the numerator) are then the same whatever the number of warps per walker.
    for (int vw = wi; vw < MRQ_VW; vw += nw) {
        acc.sA = acc.sT = acc.sD = 0.0;
        for (int u = vw; u < units; u += MRQ_VW) {
            if (cas) {
                const long long nbase = (MODE == MODE_DEBUG && nbout != nullptr) ? nb_prefix[u] : 0;
                if (u < S.cas_units) {
                    acc = cas_internal_unit<W, MODE>(S, cs.cw, nsh, u, acc, step, wid, lane, nbout, nbase, max_nb, ctr);
                    ctr.mark(1);
                } else {
                    cas_pair_unit<W, MODE>(S, cs.cw, gops, cphi, ccode, nsh, u, acc, step, wid, lane, nbout, nbase,
                                           max_nb, ctr);
                    ctr.mark(2);
                }
            } else {
                const int i0 = u * MRQ_FOIS_CH, i1 = min(total_fois, i0 + MRQ_FOIS_CH);
                acc = fois_unit<W, MODE>(S, cs.L, psin != 0.0 ? gops : nullptr, nsh, ln, c0, inv_psin, inv_psin_f,
                                         self_key, phi_self, i0, i1, acc, step, wid, lane, nbout, 0, max_nb, ctr);
                ctr.mark(7);
            }
        }
        const double sA = warp_sum(acc.sA), sT = warp_sum(acc.sT), sD = warp_sum(acc.sD);
        if (lane == 0) {
            cs.wsum[0][vw] = sA;
            cs.wsum[1][vw] = sT;
            cs.wsum[2][vw] = sD;
        }
    }
    // the race's winner: smallest clock, then smallest excitation id (order-independent)
    {
        const double bt_me = cs.rbt[threadIdx.x];
        const unsigned be_me = cs.rbexc[threadIdx.x];
        double t = bt_me;
        unsigned e = be_me;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double t2 = __shfl_xor_sync(0xffffffffu, t, o);
            const unsigned e2 = __shfl_xor_sync(0xffffffffu, e, o);
            if (t2 < t || (t2 == t && e2 < e)) {
                t = t2;
                e = e2;
            }
        }
        const unsigned win = __ballot_sync(0xffffffffu, be_me == e && bt_me == t);
        const int src = win ? __ffs(win) - 1 : 0;
        const double bpsi = cs.rbpsi[(threadIdx.x & ~31u) + src];
        if (lane == 0) {
            cs.wbt[wi] = t;
            cs.wbexc[wi] = e;
            cs.wbpsi[wi] = bpsi;
        }
    }
    ctr_flush(cs, ctr, lane);
    if (wi == 0) {
        double hnn, hdnn;
        diagonals<W>(S, cs.L, n, lane, hnn, hdnn);
        if (lane == 0) {
            cs.hnn = hnn;
            cs.hdnn = hdnn;
        }
    }
    __syncthreads();
    ctr.mark(8);
    StepOut o;
    double A = 0.0, T = 0.0, D = 0.0, bt = INFINITY, bpsi = 0.0;
    unsigned be = 0xFFFFFFFFu;
    for (int k = 0; k < MRQ_VW; k++) {
        A += cs.wsum[0][k];
        T += cs.wsum[1][k];
        D += cs.wsum[2][k];
    }
    for (int k = 0; k < nw; k++) {
        if (cs.wbt[k] < bt || (cs.wbt[k] == bt && cs.wbexc[k] < be)) {
            bt = cs.wbt[k];
            be = cs.wbexc[k];
            bpsi = cs.wbpsi[k];
        }
    }
    o.S = fabs(inv_psin) * A;
    o.hnn = cs.hnn;
    o.hdnn = cs.hdnn;
    o.EL = o.hnn + inv_psin * T;
    o.num = ln > 0 ? o.hdnn + inv_psin * D : 0.0;
    o.nnb = cas ? (long long)S.cas_nb_total : (long long)total_fois;
    o.bexc = be;
    o.bpsi = bpsi;
    return o;
}

// apply the excitation code of the race's winner to n
template <int W>
__device__ __forceinline__ void apply_code(unsigned long long (&m)[2][W], const SysDev& S, unsigned exc) {
    const int r1 = exc & 255u, r2 = (exc >> 8) & 255u, a1 = (exc >> 16) & 255u, a2 = (exc >> 24) & 255u;
    int s = r1 >= S.n;
    flip_reg<W>(m, s, r1 - s * S.n);
    s = a1 >= S.n;
    flip_reg<W>(m, s, a1 - s * S.n);
    if (r2 != r1) {
        s = r2 >= S.n;
        flip_reg<W>(m, s, r2 - s * S.n);
        s = a2 >= S.n;
        flip_reg<W>(m, s, a2 - s * S.n);
    }
}

// One walker step per block: slot blockIdx.x (or order[blockIdx.x]) of the walk set.  The step's
// contribution goes into the walker's record; k_accum adds the records into the accumulators.
template <int W, int MINB>
__global__ void __launch_bounds__(MRQ_MAXNW * 32, MINB) k_walk2(const WalkSet ws, const unsigned* __restrict__ order,
                                                             int accumulate) {
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    CtaSh& cs = *reinterpret_cast<CtaSh*>(smem_dyn);
    unsigned char* lists = smem_dyn + (sizeof(CtaSh) + 15) / 16 * 16;
    const long long s0 = blockIdx.x;
    if (s0 >= ws.nslots) return;
    const long long slot = order ? (long long)order[s0] : s0;
    int sys;
    long long local;
    slot_owner(ws, slot, sys, local);
    Walker* const walkers = ws.walkers[sys];
    {
        const int* src = reinterpret_cast<const int*>(ws.systems + sys);
        int* dst = reinterpret_cast<int*>(&cs.L.sys);
        for (int k = threadIdx.x; k < (int)(sizeof(SysDev) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
    }
    __syncthreads();
    const SysDev& S = cs.L.sys;
    Walker wk = walkers[local];
    unsigned long long n[2][W];
#pragma unroll
    for (int sg = 0; sg < 2; sg++)
#pragma unroll
        for (int w = 0; w < W; w++) n[sg][w] = wk.d[sg][w];
    int h, p;
    const long long ln = det_label<W>(S, n, h, p);
#ifdef MRQ_PHASE_TIMING
    PhCtr nc;
    nc.mark(9);
#else
    NoCtr nc;
#endif
    StepOut o;
    if (ln >= 0) o = block_local<W, MODE_STEP>(cs, lists, n, wk.psi, ln, h, p, wk.step, wk.wid, nullptr, 0, nullptr, nc);
#ifdef MRQ_PHASE_TIMING
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 10; k++) atomicAdd(&g_phase[k], (unsigned long long)nc.acc[k]);
#endif
    if (threadIdx.x != 0) return;
    wk.rl = -1;
    if (ln < 0 || !(o.S > 0.0) || o.bexc == 0xFFFFFFFFu) {
        atomicOr(S.err, ln < 0 ? MRQ_ERR_LABEL : MRQ_ERR_NOMOVE);
        walkers[local] = wk;
        return;
    }
    if (accumulate && (long long)wk.step >= S.burn_in) {
        wk.rl = ln;
        wk.rtype = 3 * h + p;
        wk.rw = 1.0 / o.S;
        wk.rEL = o.EL;
        wk.rnum = o.num;
    }
    apply_code<W>(n, S, o.bexc);
#pragma unroll
    for (int sg = 0; sg < 2; sg++)
#pragma unroll
        for (int w = 0; w < W; w++) wk.d[sg][w] = n[sg][w];
    wk.psi = o.bpsi;
    wk.step++;
    walkers[local] = wk;
}

// Accumulate the last step's walker records (Eq. 12, Eq. 16; weight w = 1/S): one warp per
// (system, group), walkers of the group in id order, label-0 (CAS) sums as warp sums in a fixed
// order and the other labels one lane at a time in lane order - the same result on every run.
__global__ void __launch_bounds__(1024) k_accum(const WalkSet ws) {
    const int sys = blockIdx.x;
    const int g = blockIdx.y * 32 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    const SysDev& S = ws.systems[sys];
    if (g >= S.G) return;
    Walker* const wk = ws.walkers[sys];
    const long long nw = ws.offsets[sys + 1] - ws.offsets[sys];
    const long long L = S.nlab;
    double n0 = 0.0, a0 = 0.0, b0 = 0.0, wsum = 0.0, esum = 0.0;
    const double c0 = S.c[0];
    for (long long base = g; base < nw; base += 32LL * S.G) {
        const long long i = base + (long long)lane * S.G;
        long long l = -1;
        double w = 0.0, EL = 0.0, num = 0.0;
        int type = 0;
        if (i < nw) {
            l = wk[i].rl;
            w = wk[i].rw;
            EL = wk[i].rEL;
            num = wk[i].rnum;
            type = wk[i].rtype;
        }
        if (l >= 0) {
            wsum += w;
            esum += w * EL;
            atomicAdd(S.type_steps + type, 1ull);
        }
        if (l == 0) {
            n0 += w / (c0 * c0);
            a0 += (w * EL) / c0;
            b0 += w / c0;
        }
        unsigned m = __ballot_sync(0xffffffffu, l > 0);
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            if (lane == src) {
                const double cl = S.c[l], c2 = cl * cl;
                const long long at = (long long)g * L + l;
                S.accN[at] += w / c2;
                S.accU[at] += (w * num) / c2;
                S.accA[at] += (w * EL) / cl;
                S.accB[at] += w / cl;
            }
            __syncwarp();
        }
    }
    n0 = warp_sum(n0);
    a0 = warp_sum(a0);
    b0 = warp_sum(b0);
    wsum = warp_sum(wsum);
    esum = warp_sum(esum);
    if (lane == 0) {
        const long long at = (long long)g * L;
        S.accN[at] += n0;
        S.accA[at] += a0;
        S.accB[at] += b0;
        S.accW[g] += wsum;
        S.accE[g] += esum;
    }
}

// local quantities of arbitrary determinants (parity): one block per determinant, the walk's code
template <int W>
__global__ void __launch_bounds__(MRQ_MAXNW * 32, 2) k_debug2(const SysDev* __restrict__ sys,
                                                              const unsigned long long* __restrict__ dets, long long ndet,
                                                              mrq_local* __restrict__ out, long long max_nb,
                                                              mrq_neighbour* __restrict__ nb, long long* nb_prefix,
                                                              int prefix_stride) {
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    CtaSh& cs = *reinterpret_cast<CtaSh*>(smem_dyn);
    unsigned char* lists = smem_dyn + (sizeof(CtaSh) + 15) / 16 * 16;
    const long long i = blockIdx.x;
    if (i >= ndet) return;
    {
        const int* src = reinterpret_cast<const int*>(sys);
        int* dst = reinterpret_cast<int*>(&cs.L.sys);
        for (int k = threadIdx.x; k < (int)(sizeof(SysDev) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
        if (threadIdx.x < 4) cs.ctr[threadIdx.x] = 0;
    }
    __syncthreads();
    const SysDev& S = cs.L.sys;
    unsigned long long n[2][W];
#pragma unroll
    for (int w = 0; w < W; w++) {
        n[0][w] = dets[i * 2 * W + w];
        n[1][w] = dets[i * 2 * W + W + w];
    }
    int h, p;
    const long long ln = det_label<W>(S, n, h, p);
    mrq_local r;
    memset(&r, 0, sizeof r);
    r.label = ln;
    r.type = 3 * h + p;
    if (ln < 0) {
        if (threadIdx.x == 0) out[i] = r;
        return;
    }
    double psin;
    NoCtr nc0;
    if (ln == 0) psin = __ldg(S.c) * hash_lookup(S, hash_key(S, active_bits<W>(S, n[0]), active_bits<W>(S, n[1])), nc0);
    else psin = __ldg(S.c + ln) * reach_back<W>(S, n, nc0);
    Ctr ctr;
    mrq_neighbour* rec = nb ? nb + i * max_nb : nullptr;
    const StepOut o = block_local<W, MODE_DEBUG>(cs, lists, n, psin, ln, h, p, 0, 0, rec, max_nb,
                                                 nb_prefix ? nb_prefix + i * (long long)prefix_stride : nullptr, ctr);
    __syncthreads();
    if (threadIdx.x == 0) {
        r.n_gathers = (long long)cs.ctr[0];
        r.n_probes = (long long)cs.ctr[1];
        r.n_candidates = (long long)cs.ctr[2];
        r.n_terms = (long long)cs.ctr[3];
        r.S = o.S;
        r.e_local = o.EL;
        r.num = o.num;
        r.h_nn = o.hnn;
        r.hd_nn = o.hdnn;
        r.psi = psin;
        r.n_neighbours = o.nnb;
        out[i] = r;
    }
}
