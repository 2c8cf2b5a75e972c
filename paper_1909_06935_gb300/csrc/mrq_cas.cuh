// Local evaluation at a CAS walker, organised by active remnant (included by mrq.cu).
//
// Every neighbour m of a CAS determinant n is n with active electrons X_a -> active holes Y_a
// and core electrons X_c -> virtual orbitals Y_v (|X_a|+|X_c| = |Y_a|+|Y_v| <= 2).  Its reach-back
// candidates k (Eq. 6-7: the reference determinants H-connected to m) are
//     k = m - (Y_v u R') + (X_c u A'),   R' active electrons of m, A' active holes of m,
// and which (R', A') occur, and phi0(k), depend only on the active remnant A_m = A_n - X_a + Y_a and
// on the counts and spins of X_c and Y_v - not on which core / virtual orbitals they are.  So the
// neighbours are processed in groups (X_a, Y_a, spins of X_c and Y_v): the warp builds the group's
// candidate list once (lanes probe distinct keys in parallel, compacted into shared memory), then
// the lanes run over the group's core / virtual orbital choices and evaluate
//     O(m) = H_nm phi0(n) + sum_{k in list} <m|H|k> phi0(k)
// in lockstep; the k = n term needs no lookup.  Every neighbour and every candidate of the plain
// enumeration is visited exactly once, so the sums are the same as in local_eval.

__device__ __forceinline__ int nsub(int cnt, int size) {
    return size == 0 ? 1 : (size == 1 ? cnt : cnt * (cnt - 1) / 2);
}

// position of the k-th (0-based) set bit of a 64-bit mask
__device__ __forceinline__ int nth_bit64(unsigned long long m, int k) {
    for (int i = 0; i < k; i++) m &= m - 1;
    return __ffsll(m) - 1;
}

// pair index -> (i < j), lexicographic among k <= 128 items, from the co-lexicographic table
// (colex[q] = i | j << 8 for q = j(j-1)/2 + i): the same map as lex_decode without a square root
__device__ __forceinline__ void lex_decode_tab(const unsigned short* __restrict__ colex, int op, int k, int& i, int& j) {
    const unsigned e = __ldg(colex + (k * (k - 1) / 2 - 1 - op));
    i = k - 1 - (int)(e >> 8);
    j = k - 1 - (int)(e & 255u);
}

// floor(x / d) for x * d < 2^32 from m = magic32(d) (m = 0 stands for d = 1)
__device__ __forceinline__ unsigned magic32(unsigned d) { return d > 1u ? 0xFFFFFFFFu / d + 1u : 0u; }
__device__ __forceinline__ unsigned div_m(unsigned x, unsigned m) { return m ? __umulhi(x, m) : x; }

// the idx-th subset of `size` (0..2) set bits of m (cnt = popcount of m), lexicographic
__device__ __forceinline__ unsigned long long subset_bits(const unsigned short* __restrict__ colex, unsigned long long m,
                                                          int cnt, int size, int idx) {
    if (size == 0) return 0ull;
    if (size == 1) return 1ull << nth_bit64(m, idx);
    int i, j;
    lex_decode_tab(colex, idx, cnt, i, j);
    return (1ull << nth_bit64(m, i)) | (1ull << nth_bit64(m, j));
}

// combined active bit (alpha bits 0..31, beta 32..63) -> spin orbital
__device__ __forceinline__ int act_so(const SysDev& S, int b) { return (b >= 32 ? S.n : 0) + S.nc + (b & 31); }

// up to two set bits of a combined active mask as sorted spin orbitals (returns the count)
__device__ __forceinline__ int act_list(const SysDev& S, unsigned long long bits, int* out) {
    int k = 0;
    while (bits) {
        int b = __ffsll(bits) - 1;
        bits &= bits - 1;
        out[k++] = act_so(S, b);
    }
    return k;
}

// number of choices of `cnt` orbitals of one space (size m) with `nal` of them alpha
__device__ __forceinline__ int shape_count(int m, int cnt, int nal) {
    if (cnt == 0) return 1;
    if (cnt == 1) return m;
    return nal == 1 ? m * m : m * (m - 1) / 2;
}

// idx-th choice of that shape as sorted spin orbitals; orbitals of the space start at `off`;
// mag = ceil(2^64 / m) (0 when m = 1) for the alpha-beta division
__device__ __forceinline__ void shape_decode(const SysDev& S, int m, int cnt, int nal, int off, int idx, int* out,
                                             unsigned long long mag) {
    if (cnt == 1) {
        out[0] = (nal ? 0 : S.n) + off + idx;
    } else if (cnt == 2) {
        if (nal == 1) {
            const int i = mag ? (int)__umul64hi((unsigned long long)idx, mag) : idx, j = idx - i * m;
            out[0] = off + i;
            out[1] = S.n + off + j;
        } else {
            int i, j;
            lex_decode_tab(S.colex, idx, m, i, j);
            const int base = (nal == 2 ? 0 : S.n) + off;
            out[0] = base + i;
            out[1] = base + j;
        }
    }
}

__device__ __forceinline__ void sort2(int* x, int k) {
    if (k == 2 && x[0] > x[1]) {
        int t = x[0];
        x[0] = x[1];
        x[1] = t;
    }
}

template <int W>
__device__ __forceinline__ void apply_exc(unsigned long long (&m)[2][W], const SysDev& S, const int* rem,
                                          const int* add, int k) {
    for (int i = 0; i < k; i++) {
        int s1 = rem[i] >= S.n, s2 = add[i] >= S.n;
        flip_reg<W>(m, s1, rem[i] - s1 * S.n);
        flip_reg<W>(m, s2, add[i] - s2 * S.n);
    }
}

// candidate code: R' and A' as combined active bit positions (7 bits each, 127 = none) and the order
#define MRQ_NONE 127u
__device__ __forceinline__ unsigned pack_cand(unsigned long long R, unsigned long long A, int rr) {
    unsigned p[4] = {MRQ_NONE, MRQ_NONE, MRQ_NONE, MRQ_NONE};
    int k = 0;
    while (R) { p[k++] = (unsigned)(__ffsll(R) - 1); R &= R - 1; }
    k = 2;
    while (A) { p[k++] = (unsigned)(__ffsll(A) - 1); A &= A - 1; }
    return p[0] | (p[1] << 7) | (p[2] << 14) | (p[3] << 21) | ((unsigned)(rr - 1) << 28);
}

// flip the sign of x when the low bit of `odd` is set (exact, no floating-point operation)
__device__ __forceinline__ double neg_if(double x, int odd) {
    return __longlong_as_double(__double_as_longlong(x) ^ ((long long)(odd & 1) << 63));
}

// the two removed (or added) spin orbitals of a candidate: `cnt` lane orbitals l0, l1 first, then
// the candidate's active orbitals from its code (bit positions b0, b1); returned sorted
__device__ __forceinline__ void merge_pair(const SysDev& S, int cnt, int l0, int l1, unsigned b0, unsigned b1,
                                           int& x0, int& x1) {
    const int c0 = act_so(S, (int)(b0 & 63u)), c1 = act_so(S, (int)(b1 & 63u));
    x0 = cnt >= 1 ? l0 : c0;
    x1 = cnt == 2 ? l1 : (cnt == 1 ? c0 : c1);
    if (x0 > x1) {
        int t = x0;
        x0 = x1;
        x1 = t;
    }
}

// <m|H|k> for a double candidate: removed = lane's virtual electrons yv + candidate's R',
// added = lane's core holes xc + candidate's A' (pairing by sorted order, spin conserving)
template <int W, class C>
__device__ __forceinline__ double dbl_elem_code(const SysDev& S, const unsigned long long (&m)[2][W], unsigned code,
                                                int nyv, int yv0, int yv1, int nxc, int xc0, int xc1, C& ctr) {
    int r1, r2, a1, a2;
    merge_pair(S, nyv, yv0, yv1, code & 127u, (code >> 7) & 127u, r1, r2);
    merge_pair(S, nxc, xc0, xc1, (code >> 14) & 127u, (code >> 21) & 127u, a1, a2);
    const int n = S.n;
    const int s_r1 = r1 >= n, s_r2 = r2 >= n;
    const int pr1 = r1 - s_r1 * n, pr2 = r2 - s_r2 * n, pa1 = a1 - (a1 >= n) * n, pa2 = a2 - (a2 >= n) * n;
    int c1 = popc_sel<W>(m, s_r1, min(pr1, pa1), max(pr1, pa1));
    int c2;
    if (s_r2 == s_r1) {
        unsigned long long t[W];
#pragma unroll
        for (int w = 0; w < W; w++) t[w] = s_r1 ? m[1][w] : m[0][w];
        flip<W>(t, pr1);
        flip<W>(t, pa1);
        c2 = popc_between<W>(t, min(pr2, pa2), max(pr2, pa2));
    } else {
        c2 = popc_sel<W>(m, s_r2, min(pr2, pa2), max(pr2, pa2));
    }
    double v = __ldg(S.eri4 + eri_idx(S, pa1, pr1, pa2, pr2));
    ctr.g();
    if (s_r1 == s_r2) {
        v -= __ldg(S.eri4 + eri_idx(S, pa1, pr2, pa2, pr1));
        ctr.g();
    }
    return neg_if(v, c1 + c2);
}

// A double candidate of a group as a signed table lookup.  With the added pair A = (A0, A1) and the
// removed pair R = (R0, R1) of m -> k ordered "candidate's active orbitals first, lane's core /
// virtual orbitals last", <m|H|k> = sgn (-1)^(piA + piR) <A0 A1||R0 R1>, where <A0 A1||R0 R1> is
// <pq||rs> (same spin), <pq|rs> (A0, R0 same spin) or -<A0 A1|R1 R0>.  Which orbital sits in which slot,
// piA, piR and the spin pattern do not depend on the lane (the classes fix the order), and sgn
// changes between lanes only by (-1)^(sum of the lane's core-hole positions): no occupied orbital lies
// between a virtual and the active block, while the core orbitals above a hole are all occupied.
// So the entry stores w = phi0(k) * (sign for the reference lane, its core parity removed) and the
// table index without the lane part; a lane adds its offset and multiplies by its own core parity.
template <int W>
__device__ __forceinline__ void dbl_entry(const SysDev& S, const unsigned long long (&mref)[2][W], int c, int v,
                                          int xc0, int xc1, int yv0, int yv1, int par_ref, unsigned long long Rb,
                                          unsigned long long Ab, double phi, double& w, unsigned& bp) {
    const int n = S.n, ne = 2 - v, nf = 2 - c;
    int rc[2] = {0, 0}, ac[2] = {0, 0};    // candidate's active orbitals, sorted
    {
        unsigned long long x = Rb;
        if (x) { rc[0] = act_so(S, __ffsll(x) - 1); x &= x - 1; }
        if (x) rc[1] = act_so(S, __ffsll(x) - 1);
        x = Ab;
        if (x) { ac[0] = act_so(S, __ffsll(x) - 1); x &= x - 1; }
        if (x) ac[1] = act_so(S, __ffsll(x) - 1);
    }
    const int A0 = nf >= 1 ? ac[0] : xc0, A1 = nf == 2 ? ac[1] : (nf == 1 ? xc0 : xc1);
    const int R0 = ne >= 1 ? rc[0] : yv0, R1 = ne == 2 ? rc[1] : (ne == 1 ? yv0 : yv1);
    const int a1 = min(A0, A1), a2 = max(A0, A1), r1 = min(R0, R1), r2 = max(R0, R1);
    const int piA = A0 > A1, piR = R0 > R1;
    // sign of the reference lane's element (pairing r1 -> a1, r2 -> a2, sequential singles on m)
    const int s_r1 = r1 >= n, s_r2 = r2 >= n;
    const int pr1 = r1 - s_r1 * n, pr2 = r2 - s_r2 * n, pa1 = a1 - (a1 >= n) * n, pa2 = a2 - (a2 >= n) * n;
    int c1 = popc_sel<W>(mref, s_r1, min(pr1, pa1), max(pr1, pa1));
    int c2;
    if (s_r2 == s_r1) {
        unsigned long long t[W];
#pragma unroll
        for (int w2 = 0; w2 < W; w2++) t[w2] = s_r1 ? mref[1][w2] : mref[0][w2];
        flip<W>(t, pr1);
        flip<W>(t, pa1);
        c2 = popc_between<W>(t, min(pr2, pa2), max(pr2, pa2));
    } else {
        c2 = popc_sel<W>(mref, s_r2, min(pr2, pa2), max(pr2, pa2));
    }
    const int sA0 = A0 >= n, sA1 = A1 >= n, sR0 = R0 >= n, sR1 = R1 >= n;
    const bool same = sA0 == sA1 && sR0 == sR1 && sA0 == sR0;
    const bool xpat = !same && sA0 != sR0;              // the allowed pairing is (A0,R1)(A1,R0)
    // strides of T[p][q][r][s] on the (core+active)^2 x (active+virtual)^2 block
    const unsigned sv = (unsigned)S.nav, sq = sv * sv, sp = sq * (unsigned)S.nca;
    const unsigned pA0 = (unsigned)(A0 - sA0 * n), pA1 = (unsigned)(A1 - sA1 * n);
    const unsigned pR0 = (unsigned)(R0 - sR0 * n - S.nc), pR1 = (unsigned)(R1 - sR1 * n - S.nc);
    unsigned base = same ? S.tab_half : 0u;
    if (nf >= 1) base += pA0 * sp;
    if (nf == 2) base += pA1 * sq;
    if (!xpat) {
        if (ne >= 1) base += pR0 * sv;
        if (ne == 2) base += pR1;
    } else {
        if (ne == 2) base += pR1 * sv;
        if (ne >= 1) base += pR0;
    }
    const int odd = c1 + c2 + piA + piR + (xpat ? 1 : 0) + par_ref;
    w = neg_if(phi, odd);
    bp = base | (xpat ? 0x80000000u : 0u);
}

// a lane's table offsets for the direct and the swapped removed-pair layouts, and its core parity
__device__ __forceinline__ void lane_offsets(const SysDev& S, int c, int v, int xc0, int xc1, int yv0, int yv1,
                                             unsigned& off_d, unsigned& off_x, int& par) {
    const unsigned sv = (unsigned)S.nav, sq = sv * sv, sp = sq * (unsigned)S.nca;
    const unsigned p0 = (unsigned)(xc0 - (xc0 >= S.n ? S.n : 0)), p1 = (unsigned)(xc1 - (xc1 >= S.n ? S.n : 0));
    const unsigned v0 = (unsigned)(yv0 - (yv0 >= S.n ? S.n : 0) - S.nc), v1 = (unsigned)(yv1 - (yv1 >= S.n ? S.n : 0) - S.nc);
    const unsigned core = c == 2 ? p0 * sp + p1 * sq : (c == 1 ? p0 * sq : 0u);
    off_d = core + (v == 2 ? v0 * sv + v1 : (v == 1 ? v0 : 0u));
    off_x = core + (v == 2 ? v1 * sv + v0 : (v == 1 ? v0 * sv : 0u));
    par = (c >= 1 ? (int)p0 : 0) + (c == 2 ? (int)p1 : 0);
}

// sum over the table-form double candidates e0, e0 + stride, ... < e1 (list order)
template <class C>
__device__ __forceinline__ double tab_sum(const SysDev& S, const double* cphi, const unsigned* ccode, int e0, int e1,
                                          int stride, unsigned off_d, unsigned off_x, C& ctr) {
#ifndef MRQ_TAB_UNROLL
#define MRQ_TAB_UNROLL 4
#endif
    double p[MRQ_TAB_UNROLL];
#pragma unroll
    for (int k = 0; k < MRQ_TAB_UNROLL; k++) p[k] = 0.0;
    int e = e0;
    for (; e + (MRQ_TAB_UNROLL - 1) * stride < e1; e += MRQ_TAB_UNROLL * stride) {
        double x[MRQ_TAB_UNROLL];
#pragma unroll
        for (int k = 0; k < MRQ_TAB_UNROLL; k++) {
            const unsigned bp = ccode[e + k * stride];
            x[k] = __ldg(S.tab + (bp & 0x7FFFFFFFu) + ((bp & 0x80000000u) ? off_x : off_d));
        }
#pragma unroll
        for (int k = 0; k < MRQ_TAB_UNROLL; k++) p[k] = fma(cphi[e + k * stride], x[k], p[k]);
        ctr.g(MRQ_TAB_UNROLL);
    }
    for (; e < e1; e += stride) {
        const unsigned bp = ccode[e];
        p[0] = fma(cphi[e], __ldg(S.tab + (bp & 0x7FFFFFFFu) + ((bp & 0x80000000u) ? off_x : off_d)), p[0]);
        ctr.g();
    }
    double t = p[0];
#pragma unroll
    for (int k = 1; k < MRQ_TAB_UNROLL; k++) t += p[k];
    return t;
}

// sum over double candidates e0, e0 + stride, ... < e1 of phi_e <m|H|k_e> (list order)
template <int W, class C>
__device__ __forceinline__ double cand_sum(const SysDev& S, const unsigned long long (&m)[2][W], const double* cphi,
                                           const unsigned* ccode, int e0, int e1, int stride, int nyv, int yv0, int yv1,
                                           int nxc, int xc0, int xc1, C& ctr) {
    double p0 = 0.0;
    for (int e = e0; e < e1; e += stride)
        p0 = fma(cphi[e], dbl_elem_code<W>(S, m, ccode[e], nyv, yv0, yv1, nxc, xc0, xc1, ctr), p0);
    return p0;
}

// The walker's single-excitation operator, for every hole y (core or active) and electron x (active
// or virtual) of one spin s:  G^s_yx(n) = hc_yx + sum_{j in act occ(n)} (yx|jj) - sum_{j in act occ_s(n)} (yj|jx)
// (n a CAS determinant: full core, empty virtuals), tabulated per walker step by the walk block
// (2 x nca x nav doubles, [s][y][x - nc]; the active-active block is not needed).  Slater-Condon
// gives, for a neighbour m = n - R + A and its single x -> y,  <k|H|m> = sign (G^s_yx(n) +
// sum_{j in A} f(j) - sum_{j in R} f(j)), f(j) = (yx|jj) - d_{s_j s} (yj|jx): the same sum as
// single_elem over occ(m), with <= 4 corrections in place of one term per occupied orbital.

// f(j) of one orbital j (spin orbital) for the single x -> y of spin sx (spatial px, py)
__device__ __forceinline__ double single_corr(const SysDev& S, int sx, int px, int py, int j) {
    const int sj = j >= S.n, pj = j - sj * S.n;
    double v = eri_g(S, py, px, pj, pj);
    if (sj == sx) v -= eri_g(S, py, pj, pj, px);
    return v;
}

// <m|H|k> for a single candidate x -> y (x: lane's virtual electron or R', y: lane's hole or A');
// with the walker's operator g (CAS walkers), from g and the corrections of m's removed (rm) and
// added (ad) orbitals relative to n (r of each); else by the full Slater-Condon sum
template <int W, class C>
__device__ __forceinline__ double sgl_elem_code(const SysDev& S, const double* g, const unsigned long long (&m)[2][W],
                                                unsigned code, int nyv, int yv0, int nxc, int xc0, int r, int rm0,
                                                int rm1, int ad0, int ad1, C& ctr) {
    const int x = nyv ? yv0 : act_so(S, (int)(code & 127u));
    const int y = nxc ? xc0 : act_so(S, (int)((code >> 14) & 127u));
    if (g == nullptr) return single_elem<W>(S, m, x, y, ctr);
    const int sx = x >= S.n, px = x - sx * S.n, py = y - sx * S.n;
    double v = g[(sx * S.nca + py) * S.nav + (px - S.nc)];
    v += single_corr(S, sx, px, py, ad0) - single_corr(S, sx, px, py, rm0);
    if (r == 2) v += single_corr(S, sx, px, py, ad1) - single_corr(S, sx, px, py, rm1);
    ctr.g(1 + 4 * r);
    return neg_if(v, popc_sel<W>(m, sx, min(px, py), max(px, py)));
}

// the cnt (1 or 2) items made of k1 "first" items (f0, f1) and then (s0, s1), sorted when cnt = 2
__device__ __forceinline__ void join_sorted(int cnt, int k1, int f0, int f1, int s0, int s1, int& x0, int& x1) {
    x0 = k1 >= 1 ? f0 : s0;
    x1 = k1 == 2 ? f1 : (k1 == 1 ? s0 : s1);
    if (cnt == 2 && x0 > x1) {
        int t = x0;
        x0 = x1;
        x1 = t;
    }
}

// neighbour (ic, iv) of a group: core holes xc, virtual electrons yv, removed / added pairs and m
template <int W>
__device__ __forceinline__ void group_neighbour(const SysDev& S, const unsigned long long (&n)[2][W], int nc, int nv,
                                                int voff, int c, int sc, int v, int sv, int ic, int iv, int ka,
                                                int xa0, int xa1, int kb, int ya0, int ya1, int r, int& xc0, int& xc1,
                                                int& yv0, int& yv1, int& rm0, int& rm1, int& ad0, int& ad1,
                                                unsigned long long (&m)[2][W]) {
    int t[2] = {0, 0}, u[2] = {0, 0};
    shape_decode(S, nc, c, sc, 0, ic, t, S.mag_c);
    shape_decode(S, nv, v, sv, voff, iv, u, S.mag_v);
    xc0 = t[0];
    xc1 = t[1];
    yv0 = u[0];
    yv1 = u[1];
    join_sorted(r, ka, xa0, xa1, xc0, xc1, rm0, rm1);
    join_sorted(r, kb, ya0, ya1, yv0, yv1, ad0, ad1);
#pragma unroll
    for (int sg = 0; sg < 2; sg++)
#pragma unroll
        for (int w = 0; w < W; w++) m[sg][w] = n[sg][w];
    {
        int s1 = rm0 >= S.n, s2 = ad0 >= S.n;
        flip_reg<W>(m, s1, rm0 - s1 * S.n);
        flip_reg<W>(m, s2, ad0 - s2 * S.n);
    }
    if (r == 2) {
        int s1 = rm1 >= S.n, s2 = ad1 >= S.n;
        flip_reg<W>(m, s1, rm1 - s1 * S.n);
        flip_reg<W>(m, s2, ad1 - s2 * S.n);
    }
}
