/*
 * Plain CPU oracle for the stochastic SC-NEVPT2(s) / SC-MRCI(s) local-estimator path of
 * Mahajan, Blunt, Sabzevari and Sharma, "Multireference configuration interaction and
 * perturbation theory without reduced density matrices" (arXiv:1909.06935).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg may load this library.  It shares no code with the CUDA path: determinants are handled
 * one orbital at a time, matrix elements come from a general Slater-Condon routine that first
 * works out the excitation between two determinants, and the reference is a sorted array
 * searched by bisection.  Everything is FP64.
 *
 * Conventions (the paper prints none of them; the textbook ones are used):
 *  - spatial orbitals 0..n-1 ordered core, active, virtual; spin orbital so = sigma*n + p
 *    (alpha sigma=0 first); |det> = prod_{alpha p asc} a+_p prod_{beta p asc} a+_p |vac>.
 *  - a+_q a_p on a determinant carries (-1)^(occupied orbitals of that spin strictly between).
 *  - chemists' integrals (pq|rs), 8-fold packed: eri[P(P(p,q),P(r,s))], P(x,y)=x(x+1)/2+y, x>=y;
 *    <ab|ij> = (ai|bj) with spin deltas.
 *  - perturber label of a determinant (Sec. II A, S_l^(k)): the set H of empty core spin
 *    orbitals and the set P of occupied virtual spin orbitals, |H|,|P| <= 2, ranked as
 *    rank(H) * nPsets + rank(P); rank(empty)=0, rank({x})=1+x, rank({x<y})=1+m+y(y-1)/2+x,
 *    m the number of spin orbitals of that space.  Label 0 is the CAS.
 *
 * Parity pins live in the test suite (closed forms, an independent second-quantised operator
 * applier, brute force over the whole determinant space on tiny inputs).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXN 128          /* spatial orbitals */

typedef struct { uint64_t w[2][2]; } det_t;   /* w[spin][word] */

typedef struct {
    int nc, na, nv, n, W;
    int nalpha, nbeta;
    double *h1;           /* n*n */
    double *eri;          /* packed */
    double e_nuc;
    int64_t nref;
    det_t *ref;           /* sorted */
    double *refc;
    int64_t *hidx;        /* open-addressing index of ref: slot -> position + 1 (0 = empty) */
    uint64_t hmask;
    double *c;            /* per label sampling coefficients */
    int64_t nlab;
    int64_t nHs, nPs;     /* numbers of hole sets and particle sets */
    /* derived at setup (Sec. II C: Dyall's H_D) */
    double norm0, e0, e_core;
    double *gamma;        /* na*na spin-summed 1-RDM of normalised phi0 */
    double *heff;         /* na*na */
    double *eps;          /* n: diagonal of the generalised Fock operator */
    double sum_eps_core;
    int64_t start;        /* index (input order) of the largest |phi0| determinant */
    det_t start_det;
    double hb_eps;        /* heat-bath cutoff of the walk's double excitations (0: exact) */
} osys;

/* ------------------------------------------------------------------ determinants */

static int occ(const det_t *d, int so, int n) {
    int s = so / n, p = so % n;
    return (int)((d->w[s][p >> 6] >> (p & 63)) & 1u);
}
static void setb(det_t *d, int so, int n) { int s = so / n, p = so % n; d->w[s][p >> 6] |= (1ull << (p & 63)); }
static void clrb(det_t *d, int so, int n) { int s = so / n, p = so % n; d->w[s][p >> 6] &= ~(1ull << (p & 63)); }

static int det_cmp(const det_t *a, const det_t *b) {
    for (int s = 0; s < 2; s++)
        for (int k = 1; k >= 0; k--) {
            if (a->w[s][k] < b->w[s][k]) return -1;
            if (a->w[s][k] > b->w[s][k]) return 1;
        }
    return 0;
}
static int det_cmp_v(const void *a, const void *b) { return det_cmp((const det_t *)a, (const det_t *)b); }

static det_t det_from_words(const osys *S, const uint64_t *x) {
    det_t d;
    memset(&d, 0, sizeof d);
    for (int k = 0; k < S->W; k++) { d.w[0][k] = x[k]; d.w[1][k] = x[S->W + k]; }
    return d;
}
static void det_to_words(const osys *S, const det_t *d, uint64_t *x) {
    for (int k = 0; k < S->W; k++) { x[k] = d->w[0][k]; x[S->W + k] = d->w[1][k]; }
}

static int orb_class(const osys *S, int p) { return p < S->nc ? 0 : (p < S->nc + S->na ? 1 : 2); }

/* ------------------------------------------------------------------ integrals */

static int64_t pidx(int64_t x, int64_t y) { return x >= y ? x * (x + 1) / 2 + y : y * (y + 1) / 2 + x; }
static double eri(const osys *S, int p, int q, int r, int s) { return S->eri[pidx(pidx(p, q), pidx(r, s))]; }
/* <ab|ij> over spin orbitals */
static double phys(const osys *S, int a, int b, int i, int j) {
    int n = S->n;
    if (a / n != i / n || b / n != j / n) return 0.0;
    return eri(S, a % n, i % n, b % n, j % n);
}

/* sign of a+_to a_from on d (same spin, from occupied, to empty) */
static int single_sign(const osys *S, const det_t *d, int from, int to) {
    int lo = from < to ? from : to, hi = from < to ? to : from, cnt = 0;
    for (int so = lo + 1; so < hi; so++) cnt += occ(d, so, S->n);
    return (cnt & 1) ? -1 : 1;
}

/* ------------------------------------------------------------------ labels (Sec. II A) */

static int64_t set_rank(int cnt, const int *x, int m) {
    if (cnt == 0) return 0;
    if (cnt == 1) return 1 + x[0];
    return 1 + m + (int64_t)x[1] * (x[1] - 1) / 2 + x[0];
}

/* holes/particles of d; returns label or -1 when |H|>2 or |P|>2.  h,p set anyway. */
static int64_t det_label(const osys *S, const det_t *d, int *h_out, int *p_out) {
    int n = S->n, nc = S->nc, nv = S->nv, off = S->nc + S->na;
    int hs[2 * MAXN], ps[2 * MAXN], h = 0, p = 0;
    for (int s = 0; s < 2; s++)
        for (int i = 0; i < nc; i++)
            if (!occ(d, s * n + i, n)) hs[h++] = s * nc + i;
    for (int s = 0; s < 2; s++)
        for (int a = 0; a < nv; a++)
            if (occ(d, s * n + off + a, n)) ps[p++] = s * nv + a;
    if (h_out) *h_out = h;
    if (p_out) *p_out = p;
    if (h > 2 || p > 2) return -1;
    return set_rank(h, hs, 2 * nc) * S->nPs + set_rank(p, ps, 2 * nv);
}

/* ------------------------------------------------------------------ reference lookup */

static uint64_t det_hash(const det_t *d) {
    uint64_t h = 0x9E3779B97F4A7C15ull;
    for (int s = 0; s < 2; s++)
        for (int w = 0; w < 2; w++) {
            h ^= d->w[s][w] + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
            h ^= h >> 31; h *= 0xBF58476D1CE4E5B9ull; h ^= h >> 29;
        }
    return h;
}

/* phi0(d): the reference coefficient of d, or 0 (hash index over the sorted list) */
static double phi0(const osys *S, const det_t *d) {
    for (uint64_t i = det_hash(d) & S->hmask;; i = (i + 1) & S->hmask) {
        int64_t k = S->hidx[i];
        if (k == 0) return 0.0;
        if (det_cmp(&S->ref[k - 1], d) == 0) return S->refc[k - 1];
    }
}

/* ------------------------------------------------------------------ Slater-Condon (H) */

/* difference lists: orbitals occupied in a but not in b */
static int diff_list(const osys *S, const det_t *a, const det_t *b, int *out, int maxc) {
    int cnt = 0;
    for (int so = 0; so < 2 * S->n; so++)
        if (occ(a, so, S->n) && !occ(b, so, S->n)) {
            if (cnt < maxc) out[cnt] = so;
            cnt++;
        }
    return cnt;
}

static double h_diag(const osys *S, const det_t *d) {
    int n = S->n;
    double e = S->e_nuc;
    for (int i = 0; i < 2 * n; i++) {
        if (!occ(d, i, n)) continue;
        e += S->h1[(i % n) * n + i % n];
        for (int j = 0; j < 2 * n; j++) {
            if (!occ(d, j, n)) continue;
            e += 0.5 * eri(S, i % n, i % n, j % n, j % n);
            if (i / n == j / n) e -= 0.5 * eri(S, i % n, j % n, j % n, i % n);
        }
    }
    return e;
}

/* <m|H|n>: general Slater-Condon rules (Szabo-Ostlund) */
static double h_elem(const osys *S, const det_t *nd, const det_t *md) {
    int rem[4], add[4], n = S->n;
    int nr = diff_list(S, nd, md, rem, 4);
    int na = diff_list(S, md, nd, add, 4);
    if (nr != na || nr > 2) return 0.0;
    if (nr == 0) return h_diag(S, nd);
    if (nr == 1) {
        int i = rem[0], a = add[0];
        if (i / n != a / n) return 0.0;
        double v = S->h1[(a % n) * n + i % n];
        for (int j = 0; j < 2 * n; j++) {
            if (!occ(nd, j, n)) continue;
            v += eri(S, a % n, i % n, j % n, j % n);
            if (j / n == i / n) v -= eri(S, a % n, j % n, j % n, i % n);
        }
        return single_sign(S, nd, i, a) * v;
    }
    /* double: rem[0]<rem[1], add[0]<add[1] (lists are ascending) */
    int i = rem[0], j = rem[1], a = add[0], b = add[1];
    if (i / n != a / n || j / n != b / n) {
        /* only possible pairing is i->b, j->a (both of one spin class) */
        if (i / n != b / n || j / n != a / n) return 0.0;
        int t = a; a = b; b = t;
    }
    det_t mid = *nd;
    int s1 = single_sign(S, &mid, i, a);
    clrb(&mid, i, n); setb(&mid, a, n);
    int s2 = single_sign(S, &mid, j, b);
    double v = (double)(s1 * s2) * (phys(S, a, b, i, j) - phys(S, a, b, j, i));
    /* heat-bath cutoff (Sec. II D): a double excitation with |<ab||ij>| below it is not generated */
    if (S->hb_eps > 0.0 && fabs(v) < S->hb_eps) v = 0.0;
    return v;
}

/* ------------------------------------------------------------------ Dyall H_D (Sec. II C) */

static int same_label_space(const osys *S, const det_t *a, const det_t *b) {
    int n = S->n;
    for (int s = 0; s < 2; s++)
        for (int p = 0; p < n; p++)
            if (orb_class(S, p) != 1 && occ(a, s * n + p, n) != occ(b, s * n + p, n)) return 0;
    return 1;
}

static double hd_diag(const osys *S, const det_t *d) {
    int n = S->n, nc = S->nc, na = S->na;
    double e = S->e_core - 2.0 * S->sum_eps_core;
    for (int so = 0; so < 2 * n; so++) {
        if (!occ(d, so, n)) continue;
        int p = so % n, cl = orb_class(S, p);
        if (cl != 1) { e += S->eps[p]; continue; }
        int t = p - nc;
        e += S->heff[t * na + t];
        for (int so2 = 0; so2 < 2 * n; so2++) {
            if (!occ(d, so2, n) || orb_class(S, so2 % n) != 1) continue;
            int u = so2 % n;
            e += 0.5 * eri(S, p, p, u, u);
            if (so / n == so2 / n) e -= 0.5 * eri(S, p, u, u, p);
        }
    }
    return e;
}

static double hd_elem(const osys *S, const det_t *nd, const det_t *md) {
    if (!same_label_space(S, nd, md)) return 0.0;
    int rem[4], add[4], n = S->n, nc = S->nc, na = S->na;
    int nr = diff_list(S, nd, md, rem, 4);
    int nad = diff_list(S, md, nd, add, 4);
    if (nr != nad || nr > 2) return 0.0;
    if (nr == 0) return hd_diag(S, nd);
    if (nr == 1) {
        int t = rem[0], u = add[0];
        if (t / n != u / n) return 0.0;
        double v = S->heff[(u % n - nc) * na + (t % n - nc)];
        for (int so = 0; so < 2 * n; so++) {
            if (!occ(nd, so, n) || orb_class(S, so % n) != 1) continue;
            v += eri(S, u % n, t % n, so % n, so % n);
            if (so / n == t / n) v -= eri(S, u % n, so % n, so % n, t % n);
        }
        return single_sign(S, nd, t, u) * v;
    }
    return h_elem(S, nd, md);   /* active-only double: same two-electron element */
}

/* ------------------------------------------------------------------ overlaps (Eq. 6-7) */

/* O(m) = <m|H|phi0> for m outside the CAS: the determinants k of phi0 reachable from m must
 * have a full core and empty virtuals, so the excitation m->k removes every virtual electron
 * of m plus active electrons, and fills every core hole plus active holes (Sec. II D). */
static double overlap_foism(const osys *S, const det_t *m, int64_t *terms) {
    int n = S->n, rp[2 * MAXN], ap[2 * MAXN], nrp = 0, nap = 0, h = 0, p = 0;
    for (int so = 0; so < 2 * n; so++) {
        int cl = orb_class(S, so % n), o = occ(m, so, n);
        if (o && cl != 0) rp[nrp++] = so;          /* removable: active or virtual electron */
        if (!o && cl != 2) ap[nap++] = so;         /* fillable: core or active hole */
        if (!o && cl == 0) h++;
        if (o && cl == 2) p++;
    }
    double acc = 0.0;
    /* singles */
    if (h <= 1 && p <= 1)
        for (int x = 0; x < nrp; x++)
            for (int y = 0; y < nap; y++) {
                int r = rp[x], a = ap[y];
                if (r / n != a / n) continue;
                if (p == 1 && orb_class(S, r % n) != 2) continue;
                if (h == 1 && orb_class(S, a % n) != 0) continue;
                det_t k = *m; clrb(&k, r, n); setb(&k, a, n);
                double c = phi0(S, &k);
                if (c != 0.0) { acc += h_elem(S, m, &k) * c; if (terms) (*terms)++; }
            }
    /* doubles */
    for (int x1 = 0; x1 < nrp; x1++)
        for (int x2 = x1 + 1; x2 < nrp; x2++) {
            int nvirt = (orb_class(S, rp[x1] % n) == 2) + (orb_class(S, rp[x2] % n) == 2);
            if (nvirt != p) continue;
            for (int y1 = 0; y1 < nap; y1++)
                for (int y2 = y1 + 1; y2 < nap; y2++) {
                    int ncore = (orb_class(S, ap[y1] % n) == 0) + (orb_class(S, ap[y2] % n) == 0);
                    if (ncore != h) continue;
                    int sa = (rp[x1] / n == 0) + (rp[x2] / n == 0);
                    int sb = (ap[y1] / n == 0) + (ap[y2] / n == 0);
                    if (sa != sb) continue;
                    det_t k = *m;
                    clrb(&k, rp[x1], n); clrb(&k, rp[x2], n); setb(&k, ap[y1], n); setb(&k, ap[y2], n);
                    double c = phi0(S, &k);
                    if (c != 0.0) { acc += h_elem(S, m, &k) * c; if (terms) (*terms)++; }
                }
        }
    return acc;
}

/* <m|psi_s> = c_0 phi0(m) in the CAS, c_{l_m} O(m) in the FOIS, 0 outside (Eq. 6-7, 17) */
static double psi_s_t(const osys *S, const det_t *m, double *o_out, int64_t *terms) {
    int h, p;
    int64_t l = det_label(S, m, &h, &p);
    if (l < 0) { if (o_out) *o_out = 0.0; return 0.0; }
    if (l == 0) { double v = phi0(S, m); if (o_out) *o_out = v; return S->c[0] * v; }
    double o = overlap_foism(S, m, terms);
    if (o_out) *o_out = o;
    return S->c[l] * o;
}
static double psi_s(const osys *S, const det_t *m, double *o_out) { return psi_s_t(S, m, o_out, NULL); }

/* ------------------------------------------------------------------ Philox4x32-10
 * Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11). */

static void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void oracle_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out) { philox4x32_10(ctr, key, out); }

/* threads of the parallel regions that follow (0 or less: the OpenMP default) */
/* heat-bath cutoff of the walk (Sec. II D): double excitations with |<ab||ij>| < eps are dropped
 * from every later neighbour list, overlap and brute-force sum; E0 and the set-up stay exact */
void oracle_set_hb_eps(void *h, double eps) {
    ((osys *)h)->hb_eps = eps > 0.0 ? eps : 0.0;
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    else omp_set_num_threads(omp_get_num_procs());
#else
    (void)n;
#endif
}

/* canonical excitation id: removed so r1<=r2, added a1<=a2 (singles repeat the orbital) */
static uint32_t exc_id(int r1, int r2, int a1, int a2) {
    return (uint32_t)r1 | ((uint32_t)r2 << 8) | ((uint32_t)a1 << 16) | ((uint32_t)a2 << 24);
}

/* exponential clock of the competing-exponentials (first-reaction) form of Gillespie's
 * algorithm: t = -ln(u)/Gamma, u in (0,1] from 53 bits of Philox(seed; exc, step, walker, 0) */
static double race_clock(uint64_t seed, uint32_t exc, uint32_t step, uint32_t walker, double rate) {
    uint32_t ctr[4] = {exc, step, walker, 0u}, key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)}, o[4];
    philox4x32_10(ctr, key, o);
    uint64_t k = ((((uint64_t)o[0]) << 32) | o[1]) >> 11;
    double u = (double)(k + 1) * (1.0 / 9007199254740992.0);
    return -log(u) / rate;
}

/* ------------------------------------------------------------------ local quantities */

typedef struct {
    double S, EL, num, Hnn, HDnn, psi_n;
    int64_t terms;      /* products H_mk phi0(k) summed into the neighbours' overlaps */
    int64_t label;
    int type;
    int64_t nnb;
    det_t next;
    double next_psi;
    uint32_t next_exc;
} local_t;

/* All quantities of one walker step at determinant d (Eq. 5, Eq. 16, Sec. II D), with the
 * move picked by the exponential race when seed/step/walker are given (do_move != 0).
 * Neighbours: every single and double of d whose image m has |H|<=2, |P|<=2. */
static void local_eval(const osys *S, const det_t *d, int do_move, uint64_t seed, uint32_t step,
                       uint32_t walker, local_t *L, int64_t max_nb, uint64_t *nb_dets, double *nb_vals,
                       uint32_t *nb_exc) {
    int n = S->n, h, p;
    memset(L, 0, sizeof *L);
    L->label = det_label(S, d, &h, &p);
    L->type = 3 * h + p;
    double on;
    L->psi_n = psi_s(S, d, &on);
    L->Hnn = h_diag(S, d);
    L->HDnn = (L->label >= 0) ? hd_diag(S, d) : 0.0;
    double sumH = 0.0, sumHD = 0.0, Ssum = 0.0, best = INFINITY;
    int64_t nnb = 0, terms = 0, rec = 0;     /* rec: neighbours recorded (serial when recording) */
    int occl[2 * MAXN], empl[2 * MAXN], no = 0, ne = 0;
    for (int so = 0; so < 2 * n; so++) { if (occ(d, so, n)) occl[no++] = so; else empl[ne++] = so; }
    /* without a neighbour list the sums may run in parallel over the first removed electron (the
     * sums then add in another order; the race winner is the same: smallest clock, then id) */
    const int par = (nb_dets == NULL);
    for (int kind = 1; kind <= 2; kind++) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) if (par) reduction(+ : sumH, sumHD, Ssum, nnb, terms)
#endif
        for (int x1 = 0; x1 < no; x1++) {
            double tbest = INFINITY, tpsi = 0.0;
            uint32_t tid = 0;
            det_t tnext = *d;
            for (int x2 = (kind == 1 ? x1 : x1 + 1); x2 < (kind == 1 ? x1 + 1 : no); x2++)
                for (int y1 = 0; y1 < ne; y1++)
                    for (int y2 = (kind == 1 ? y1 : y1 + 1); y2 < (kind == 1 ? y1 + 1 : ne); y2++) {
                        int r1 = occl[x1], r2 = occl[x2], a1 = empl[y1], a2 = empl[y2];
                        int sr = (r1 / n == 0) + (kind == 2 ? (r2 / n == 0) : 0);
                        int sa = (a1 / n == 0) + (kind == 2 ? (a2 / n == 0) : 0);
                        if (sr != sa) continue;
                        det_t m = *d;
                        clrb(&m, r1, n); setb(&m, a1, n);
                        if (kind == 2) { clrb(&m, r2, n); setb(&m, a2, n); }
                        int64_t lm = det_label(S, &m, NULL, NULL);
                        if (lm < 0) continue;
                        double o, ps = psi_s_t(S, &m, &o, &terms);
                        double hnm = h_elem(S, d, &m);
                        double hd = (L->label > 0 && lm == L->label) ? hd_elem(S, d, &m) : 0.0;
                        double ratio = (L->psi_n != 0.0) ? ps / L->psi_n : 0.0;
                        double gam = fabs(hnm * ratio);
                        sumH += hnm * ratio;
                        sumHD += hd * ratio;
                        Ssum += gam;
                        uint32_t id = exc_id(r1, r2, a1, a2);
                        if (nb_dets && rec < max_nb) {
                            int64_t k = rec++;
                            det_to_words(S, &m, nb_dets + k * 2 * S->W);
                            nb_vals[k * 5 + 0] = hnm;
                            nb_vals[k * 5 + 1] = hd;
                            nb_vals[k * 5 + 2] = o;
                            nb_vals[k * 5 + 3] = ps;
                            nb_vals[k * 5 + 4] = gam;
                            nb_exc[k] = id;
                        }
                        nnb++;
                        if (do_move && gam > 0.0) {
                            double t = race_clock(seed, id, step, walker, gam);
                            if (t < tbest || (t == tbest && id < tid)) {
                                tbest = t; tnext = m; tpsi = ps; tid = id;
                            }
                        }
                    }
            if (tbest < INFINITY) {
#ifdef _OPENMP
#pragma omp critical(oracle_race)
#endif
                {
                    if (tbest < best || (tbest == best && tid < L->next_exc)) {
                        best = tbest; L->next = tnext; L->next_psi = tpsi; L->next_exc = tid;
                    }
                }
            }
        }
    }
    L->S = Ssum;
    L->nnb = nnb;
    L->terms = terms;
    L->EL = L->Hnn + sumH;
    L->num = (L->label > 0) ? L->HDnn + sumHD : 0.0;
}

/* ------------------------------------------------------------------ setup (Sec. II C) */

static int setup(osys *S) {
    int n = S->n, nc = S->nc, na = S->na;
    /* largest |phi0| determinant in input order was recorded by the caller */
    double norm = 0.0, num = 0.0;
    int nn = na > 0 ? na * na : 1;
    double *g = calloc((size_t)nn, sizeof(double));
    S->gamma = g;
    /* active spin orbitals: the only ones a CAS-internal excitation touches */
    int act[2 * MAXN], nact = 0;
    for (int so = 0; so < 2 * n; so++)
        if (orb_class(S, so % n) == 1) act[nact++] = so;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : norm, num) reduction(+ : g[:nn])
#endif
    for (int64_t k = 0; k < S->nref; k++) {
        const det_t *d = &S->ref[k];
        double ck = S->refc[k];
        norm += ck * ck;
        num += ck * ck * h_diag(S, d);
        for (int x = 0; x < nact; x++)
            if (occ(d, act[x], n)) g[(act[x] % n - nc) * na + (act[x] % n - nc)] += ck * ck;
        /* active singles and doubles of d that stay in the CAS */
        for (int x1 = 0; x1 < nact; x1++) {
            int r1 = act[x1];
            if (!occ(d, r1, n)) continue;
            for (int y1 = 0; y1 < nact; y1++) {
                int a1 = act[y1];
                if (occ(d, a1, n) || a1 / n != r1 / n) continue;
                det_t m = *d; clrb(&m, r1, n); setb(&m, a1, n);
                double cm = phi0(S, &m);
                if (cm == 0.0) continue;
                num += ck * h_elem(S, d, &m) * cm;
                /* gamma_{a r} += <m| a+_a a_r |d> c_m c_d */
                g[(a1 % n - nc) * na + (r1 % n - nc)] += single_sign(S, d, r1, a1) * cm * ck;
            }
        }
        for (int x1 = 0; x1 < nact; x1++)
            for (int x2 = x1 + 1; x2 < nact; x2++) {
                int r1 = act[x1], r2 = act[x2];
                if (!occ(d, r1, n) || !occ(d, r2, n)) continue;
                for (int y1 = 0; y1 < nact; y1++)
                    for (int y2 = y1 + 1; y2 < nact; y2++) {
                        int a1 = act[y1], a2 = act[y2];
                        if (occ(d, a1, n) || occ(d, a2, n)) continue;
                        if ((r1 / n == 0) + (r2 / n == 0) != (a1 / n == 0) + (a2 / n == 0)) continue;
                        det_t m = *d;
                        clrb(&m, r1, n); clrb(&m, r2, n); setb(&m, a1, n); setb(&m, a2, n);
                        double cm = phi0(S, &m);
                        if (cm != 0.0) num += ck * h_elem(S, d, &m) * cm;
                    }
            }
    }
    S->norm0 = norm;
    S->e0 = num / norm;
    for (int i = 0; i < na * na; i++) S->gamma[i] /= norm;
    /* core energy and core-averaged active one-electron operator */
    S->e_core = S->e_nuc;
    for (int i = 0; i < nc; i++) {
        S->e_core += 2.0 * S->h1[i * n + i];
        for (int j = 0; j < nc; j++) S->e_core += 2.0 * eri(S, i, i, j, j) - eri(S, i, j, j, i);
    }
    S->heff = calloc((size_t)(na > 0 ? na * na : 1), sizeof(double));
    for (int t = 0; t < na; t++)
        for (int u = 0; u < na; u++) {
            int pt = nc + t, pu = nc + u;
            double v = S->h1[pt * n + pu];
            for (int i = 0; i < nc; i++) v += 2.0 * eri(S, pt, pu, i, i) - eri(S, pt, i, i, pu);
            S->heff[t * na + u] = v;
        }
    /* generalised Fock diagonal */
    S->eps = calloc((size_t)n, sizeof(double));
    S->sum_eps_core = 0.0;
    for (int p = 0; p < n; p++) {
        double v = S->h1[p * n + p];
        for (int i = 0; i < nc; i++) v += 2.0 * eri(S, p, p, i, i) - eri(S, p, i, i, p);
        for (int t = 0; t < na; t++)
            for (int u = 0; u < na; u++)
                v += S->gamma[t * na + u] * (eri(S, p, p, nc + t, nc + u) - 0.5 * eri(S, p, nc + t, nc + u, p));
        S->eps[p] = v;
        if (p < nc) S->sum_eps_core += v;
    }
    return 0;
}

/* ------------------------------------------------------------------ exported API */

void oracle_free(void *h) {
    osys *S = (osys *)h;
    if (!S) return;
    free(S->h1); free(S->eri); free(S->ref); free(S->refc); free(S->c);
    free(S->gamma); free(S->heff); free(S->eps); free(S->hidx);
    free(S);
}

/* status: 0 ok, -1 bad sizes, -2 bad reference determinant */
void *oracle_create(int nc, int na, int nv, int nalpha, int nbeta, const double *h1, const double *eri_in,
                    double e_nuc, int64_t nref, const uint64_t *dets, const double *coeffs,
                    const double *c, int64_t nlab, int *status) {
    int n = nc + na + nv;
    *status = 0;
    if (n <= 0 || n > MAXN || nref <= 0) { *status = -1; return NULL; }
    osys *S = calloc(1, sizeof(osys));
    S->nc = nc; S->na = na; S->nv = nv; S->n = n; S->W = (n + 63) / 64;
    S->nalpha = nalpha; S->nbeta = nbeta; S->e_nuc = e_nuc;
    S->nHs = 1 + 2 * nc + (int64_t)(2 * nc) * (2 * nc - 1) / 2;
    S->nPs = 1 + 2 * nv + (int64_t)(2 * nv) * (2 * nv - 1) / 2;
    if (nlab != S->nHs * S->nPs) { *status = -1; free(S); return NULL; }
    int64_t npair = (int64_t)n * (n + 1) / 2, neri = npair * (npair + 1) / 2;
    S->h1 = malloc(sizeof(double) * n * n); memcpy(S->h1, h1, sizeof(double) * n * n);
    S->eri = malloc(sizeof(double) * neri); memcpy(S->eri, eri_in, sizeof(double) * neri);
    S->c = malloc(sizeof(double) * nlab); memcpy(S->c, c, sizeof(double) * nlab);
    S->nlab = nlab;
    S->nref = nref;
    S->ref = malloc(sizeof(det_t) * nref);
    S->refc = malloc(sizeof(double) * nref);
    double bestc = -1.0;
    for (int64_t k = 0; k < nref; k++) {
        det_t d = det_from_words(S, dets + k * 2 * S->W);
        int h, p, cnt[2] = {0, 0};
        det_label(S, &d, &h, &p);
        for (int so = 0; so < 2 * n; so++) cnt[so / n] += occ(&d, so, n);
        if (h || p || cnt[0] != nalpha || cnt[1] != nbeta) { *status = -2; }
        if (fabs(coeffs[k]) > bestc) { bestc = fabs(coeffs[k]); S->start = k; S->start_det = d; }
    }
    if (*status) { free(S->h1); free(S->eri); free(S->c); free(S->ref); free(S->refc); free(S); return NULL; }
    /* sort (det, coeff) pairs by det for bisection */
    int64_t *ord = malloc(sizeof(int64_t) * nref);
    det_t *tmp = malloc(sizeof(det_t) * nref);
    for (int64_t k = 0; k < nref; k++) tmp[k] = det_from_words(S, dets + k * 2 * S->W);
    /* simple insertion-free approach: sort an index array with a det comparator */
    for (int64_t k = 0; k < nref; k++) ord[k] = k;
    /* qsort on a packed array of (det,index) */
    typedef struct { det_t d; int64_t i; } di_t;
    di_t *arr = malloc(sizeof(di_t) * nref);
    for (int64_t k = 0; k < nref; k++) { arr[k].d = tmp[k]; arr[k].i = k; }
    qsort(arr, (size_t)nref, sizeof(di_t), det_cmp_v);   /* det_t is the first member */
    for (int64_t k = 0; k < nref; k++) { S->ref[k] = arr[k].d; S->refc[k] = coeffs[arr[k].i]; }
    for (int64_t k = 1; k < nref; k++)
        if (det_cmp(&S->ref[k - 1], &S->ref[k]) == 0) *status = -3;   /* duplicate determinant */
    free(arr); free(tmp); free(ord);
    if (*status) { oracle_free(S); return NULL; }
    uint64_t cap = 1;
    while (cap < 2 * (uint64_t)nref) cap <<= 1;
    S->hmask = cap - 1;
    S->hidx = calloc(cap, sizeof(int64_t));
    for (int64_t k = 0; k < nref; k++) {
        uint64_t i = det_hash(&S->ref[k]) & S->hmask;
        while (S->hidx[i]) i = (i + 1) & S->hmask;
        S->hidx[i] = k + 1;
    }
    setup(S);
    return S;
}

/* out: e0, norm0, e_core, sum_eps_core, start index; eps[n], gamma[na*na], heff[na*na] */
void oracle_setup_info(void *h, double *out, double *eps, double *gamma, double *heff) {
    osys *S = (osys *)h;
    out[0] = S->e0; out[1] = S->norm0; out[2] = S->e_core; out[3] = S->sum_eps_core; out[4] = (double)S->start;
    if (eps) memcpy(eps, S->eps, sizeof(double) * S->n);
    if (gamma && S->na) memcpy(gamma, S->gamma, sizeof(double) * S->na * S->na);
    if (heff && S->na) memcpy(heff, S->heff, sizeof(double) * S->na * S->na);
}

int64_t oracle_label(void *h, const uint64_t *x, int *hp) {
    osys *S = (osys *)h;
    det_t d = det_from_words(S, x);
    return det_label(S, &d, &hp[0], &hp[1]);
}

double oracle_h(void *h, const uint64_t *a, const uint64_t *b) {
    osys *S = (osys *)h;
    det_t x = det_from_words(S, a), y = det_from_words(S, b);
    return h_elem(S, &x, &y);
}

double oracle_hd(void *h, const uint64_t *a, const uint64_t *b) {
    osys *S = (osys *)h;
    det_t x = det_from_words(S, a), y = det_from_words(S, b);
    return hd_elem(S, &x, &y);
}

/* psi_s(m) and, in *o, phi0(m) (CAS) or O(m) (FOIS) */
double oracle_psi(void *h, const uint64_t *x, double *o) {
    osys *S = (osys *)h;
    det_t d = det_from_words(S, x);
    return psi_s(S, &d, o);
}

/* local quantities of one determinant.
 * out[0..9] = S, E_L, num, H_nn, HD_nn, psi_n, label, type, n_neighbours, reach-back terms
 * per neighbour k: dets[k*2W..], vals[k*5..] = H_nm, HD_nm, O(m)|phi0(m), psi_s(m), Gamma, exc[k] */
int64_t oracle_local(void *h, const uint64_t *x, double *out, int64_t max_nb, uint64_t *nb_dets,
                     double *nb_vals, uint32_t *nb_exc) {
    osys *S = (osys *)h;
    det_t d = det_from_words(S, x);
    local_t L;
    local_eval(S, &d, 0, 0, 0, 0, &L, max_nb, nb_dets, nb_vals, nb_exc);
    out[0] = L.S; out[1] = L.EL; out[2] = L.num; out[3] = L.Hnn; out[4] = L.HDnn; out[5] = L.psi_n;
    out[6] = (double)L.label; out[7] = (double)L.type; out[8] = (double)L.nnb; out[9] = (double)L.terms;
    return L.nnb;
}

/* The neighbour excitations of x (every spin-conserving single and double whose image m has
 * |H| <= 2 and |P| <= 2, as in local_eval), ids exc_id(r1, r2, a1, a2) in local_eval's order; at
 * most max are written.  Returns the count.  No overlaps are evaluated, so this is fast enough to
 * list the millions of neighbours of a large determinant. */
int64_t oracle_neighbour_ids(void *h, const uint64_t *x, int64_t max, uint32_t *ids) {
    osys *S = (osys *)h;
    const det_t d = det_from_words(S, x);
    const int n = S->n;
    int occl[2 * MAXN], empl[2 * MAXN], no = 0, ne = 0;
    for (int so = 0; so < 2 * n; so++) { if (occ(&d, so, n)) occl[no++] = so; else empl[ne++] = so; }
    int64_t cnt = 0;
    for (int kind = 1; kind <= 2; kind++)
        for (int x1 = 0; x1 < no; x1++)
            for (int x2 = (kind == 1 ? x1 : x1 + 1); x2 < (kind == 1 ? x1 + 1 : no); x2++)
                for (int y1 = 0; y1 < ne; y1++)
                    for (int y2 = (kind == 1 ? y1 : y1 + 1); y2 < (kind == 1 ? y1 + 1 : ne); y2++) {
                        int r1 = occl[x1], r2 = occl[x2], a1 = empl[y1], a2 = empl[y2];
                        int sr = (r1 / n == 0) + (kind == 2 ? (r2 / n == 0) : 0);
                        int sa = (a1 / n == 0) + (kind == 2 ? (a2 / n == 0) : 0);
                        if (sr != sa) continue;
                        det_t m = d;
                        clrb(&m, r1, n); setb(&m, a1, n);
                        if (kind == 2) { clrb(&m, r2, n); setb(&m, a2, n); }
                        if (det_label(S, &m, NULL, NULL) < 0) continue;
                        if (cnt < max) ids[cnt] = exc_id(r1, r2, a1, a2);
                        cnt++;
                    }
    return cnt;
}

/* The per-neighbour quantities of local_eval for a given list of neighbours of x (ids as above):
 * dets[k*2W..] = m, vals[k*5..] = H_nm, (H_D)_nm, O(m) | phi0(m), psi_s(m), Gamma_nm.  The
 * neighbours are independent, so they are evaluated in parallel.  Returns 0, or -1 when an id is
 * not a neighbour of x (a removed orbital empty, an added one occupied, spin not conserved, or an
 * image outside CAS + FOIS). */
int oracle_neighbours(void *h, const uint64_t *x, int64_t nid, const uint32_t *ids, uint64_t *dets,
                      double *vals) {
    osys *S = (osys *)h;
    const det_t d = det_from_words(S, x);
    const int n = S->n;
    int hx, px;
    const int64_t lx = det_label(S, &d, &hx, &px);
    double on;
    const double psi_n = psi_s(S, &d, &on);
    int bad = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) reduction(| : bad)
#endif
    for (int64_t k = 0; k < nid; k++) {
        const int r1 = ids[k] & 255u, r2 = (ids[k] >> 8) & 255u, a1 = (ids[k] >> 16) & 255u, a2 = (ids[k] >> 24) & 255u;
        const int single = (r1 == r2);
        if (r1 >= 2 * n || r2 >= 2 * n || a1 >= 2 * n || a2 >= 2 * n || (single != (a1 == a2)) ||
            !occ(&d, r1, n) || !occ(&d, r2, n) || occ(&d, a1, n) || occ(&d, a2, n) ||
            (r1 / n == 0) + (single ? 0 : (r2 / n == 0)) != (a1 / n == 0) + (single ? 0 : (a2 / n == 0))) {
            bad = 1;
            continue;
        }
        det_t m = d;
        clrb(&m, r1, n); setb(&m, a1, n);
        if (!single) { clrb(&m, r2, n); setb(&m, a2, n); }
        const int64_t lm = det_label(S, &m, NULL, NULL);
        if (lm < 0) { bad = 1; continue; }
        double o;
        const double ps = psi_s(S, &m, &o);
        const double hnm = h_elem(S, &d, &m);
        const double hd = (lx > 0 && lm == lx) ? hd_elem(S, &d, &m) : 0.0;
        const double ratio = (psi_n != 0.0) ? ps / psi_n : 0.0;
        det_to_words(S, &m, dets + k * 2 * S->W);
        vals[k * 5 + 0] = hnm;
        vals[k * 5 + 1] = hd;
        vals[k * 5 + 2] = o;
        vals[k * 5 + 3] = ps;
        vals[k * 5 + 4] = fabs(hnm * ratio);
    }
    return bad ? -1 : 0;
}

/* One exponential-race move from x: writes the chosen determinant and returns its exc id. */
uint32_t oracle_move(void *h, const uint64_t *x, uint64_t seed, uint32_t step, uint32_t walker,
                     uint64_t *next, double *out) {
    osys *S = (osys *)h;
    det_t d = det_from_words(S, x);
    local_t L;
    local_eval(S, &d, 1, seed, step, walker, &L, 0, NULL, NULL, NULL);
    det_to_words(S, &L.next, next);
    out[0] = L.S; out[1] = L.EL; out[2] = L.num; out[3] = L.next_psi;
    return L.next_exc;
}

/* Continuous-time Monte Carlo (Sec. II B, ref. Gillespie): walker w starts at the largest
 * |phi0| determinant; each step evaluates the local quantities, accumulates with weight
 * 1/S (expected residence time) after burn-in into group g = w mod G, then moves.
 *   accN[g*nlab + l] += w / c_l^2         (norm estimator, Eq. 16; l = 0 is the CAS)
 *   accU[g*nlab + l] += w num / c_l^2     (H_D numerator, Eq. 16; l > 0)
 *   accW[g] += w, accE[g] += w E_L        (Eq. 4)
 *   type_steps[t] += 1 for the walker's type t = 3h + p
 *   accA[g*nlab + l] += w E_L / c_l, accB[g*nlab + l] += w / c_l   (optional; the SC-MRCI(s)
 *       energy gradient, Eq. 8-9: <n|psi_l>/<n|psi> = delta_{l,l_n} / c_l)
 * traj (optional) receives the determinant after every step (nwalk x nsteps x 2W words).
 * Returns 0, or -4 when a walker has no move (S = 0). */
int oracle_sample(void *h, int64_t nwalk, int64_t nsteps, int64_t burn, uint64_t seed, int G,
                  int nthreads, double *accN, double *accU, double *accW, double *accE,
                  int64_t *type_steps, double *accA, double *accB, uint64_t *traj) {
    osys *S = (osys *)h;
    int64_t nrec = nsteps > burn ? nsteps - burn : 0;
    int64_t tot = nwalk * nrec;
    int64_t *rl = malloc(sizeof(int64_t) * (tot ? tot : 1));
    int *rt = malloc(sizeof(int) * (tot ? tot : 1));
    double *rw = malloc(sizeof(double) * (tot ? tot : 1));
    double *rn = malloc(sizeof(double) * (tot ? tot : 1));
    double *re = malloc(sizeof(double) * (tot ? tot : 1));
    int bad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t w = 0; w < nwalk; w++) {
        det_t d = S->start_det;
        for (int64_t s = 0; s < nsteps; s++) {
            local_t L;
            local_eval(S, &d, 1, seed, (uint32_t)s, (uint32_t)w, &L, 0, NULL, NULL, NULL);
            if (!(L.S > 0.0)) { bad = 1; break; }
            if (s >= burn) {
                int64_t r = w * nrec + (s - burn);
                rl[r] = L.label; rt[r] = L.type; rw[r] = 1.0 / L.S; rn[r] = L.num; re[r] = L.EL;
            }
            d = L.next;
            if (traj) det_to_words(S, &d, traj + (w * nsteps + s) * 2 * S->W);
        }
    }
    if (!bad)
        for (int64_t w = 0; w < nwalk; w++) {
            int g = (int)(w % G);
            for (int64_t s = 0; s < nrec; s++) {
                int64_t r = w * nrec + s, l = rl[r];
                double c2 = S->c[l] * S->c[l];
                accN[g * S->nlab + l] += rw[r] / c2;
                if (l > 0) accU[g * S->nlab + l] += rw[r] * rn[r] / c2;
                accW[g] += rw[r];
                accE[g] += rw[r] * re[r];
                if (accA) accA[g * S->nlab + l] += rw[r] * re[r] / S->c[l];
                if (accB) accB[g * S->nlab + l] += rw[r] / S->c[l];
                type_steps[rt[r]] += 1;
            }
        }
    free(rl); free(rt); free(rw); free(rn); free(re);
    return bad ? -4 : 0;
}

/* One walker (id `walker`) from the start determinant for nsteps steps; traj receives the
 * determinant after every step (nsteps x 2W words).  Returns 0, or -4 when it has no move. */
int oracle_walk_one(void *h, uint32_t walker, int64_t nsteps, uint64_t seed, uint64_t *traj) {
    osys *S = (osys *)h;
    det_t d = S->start_det;
    for (int64_t s = 0; s < nsteps; s++) {
        local_t L;
        local_eval(S, &d, 1, seed, (uint32_t)s, walker, &L, 0, NULL, NULL, NULL);
        if (!(L.S > 0.0)) return -4;
        d = L.next;
        det_to_words(S, &d, traj + s * 2 * S->W);
    }
    return 0;
}

/* ------------------------------------------------------------------ brute force (tiny systems)
 * Deterministic strongly contracted quantities by summation over the whole FOIS:
 *   v_l = P_l H phi0 (Eq. 2): apply H to every reference determinant, bucket by label;
 *   N_l = <v_l|v_l>, D_l = <v_l|H_D|v_l> (Eq. 14 numerator), and for the sampling function
 *   psi_s = c_0 phi0 + sum_l c_l v_l: <psi_s|psi_s> and <psi_s|H|psi_s>.
 * Sizes: Nl[nlab], Dl[nlab], out[0] = <psi_s|psi_s>, out[1] = <psi_s|H|psi_s>, out[2] = FOIS size.
 * Hll (optional, nlab x nlab row-major) receives the SC-MRCI(s) Hamiltonian in the basis of the
 * strongly contracted states, Hll[l][l'] = <v_l|H|v_l'> with v_0 = phi0 (Sec. II B); their
 * overlap matrix is diagonal, diag(Nl), because different labels never share a determinant. */

typedef struct { det_t d; double v; } dv_t;

static int64_t find_dv(const dv_t *a, int64_t n, const det_t *d) {
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        int c = det_cmp(&a[mid].d, d);
        if (c == 0) return mid;
        if (c < 0) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

int oracle_brute(void *h, double *Nl, double *Dl, double *out, double *Hll) {
    osys *S = (osys *)h;
    int n = S->n;
    /* 1. collect every determinant H-connected to a reference determinant, outside the CAS */
    int64_t cap = 1 << 16, cnt = 0;
    dv_t *buf = malloc(sizeof(dv_t) * cap);
    for (int64_t k = 0; k < S->nref; k++) {
        const det_t *d = &S->ref[k];
        int occl[2 * MAXN], empl[2 * MAXN], no = 0, ne = 0;
        for (int so = 0; so < 2 * n; so++) { if (occ(d, so, n)) occl[no++] = so; else empl[ne++] = so; }
        for (int kind = 1; kind <= 2; kind++)
            for (int x1 = 0; x1 < no; x1++)
                for (int x2 = (kind == 1 ? x1 : x1 + 1); x2 < (kind == 1 ? x1 + 1 : no); x2++)
                    for (int y1 = 0; y1 < ne; y1++)
                        for (int y2 = (kind == 1 ? y1 : y1 + 1); y2 < (kind == 1 ? y1 + 1 : ne); y2++) {
                            det_t m = *d;
                            clrb(&m, occl[x1], n); setb(&m, empl[y1], n);
                            if (kind == 2) { clrb(&m, occl[x2], n); setb(&m, empl[y2], n); }
                            int hh, pp;
                            int64_t l = det_label(S, &m, &hh, &pp);
                            if (l <= 0) continue;
                            double v = h_elem(S, d, &m) * S->refc[k];
                            if (cnt == cap) { cap *= 2; buf = realloc(buf, sizeof(dv_t) * cap); }
                            buf[cnt].d = m; buf[cnt].v = v; cnt++;
                        }
    }
    qsort(buf, (size_t)cnt, sizeof(dv_t), det_cmp_v);
    /* merge duplicates: O(m) = sum over reference determinants */
    int64_t u = 0;
    for (int64_t i = 0; i < cnt; i++) {
        if (u > 0 && det_cmp(&buf[u - 1].d, &buf[i].d) == 0) buf[u - 1].v += buf[i].v;
        else buf[u++] = buf[i];
    }
    memset(Nl, 0, sizeof(double) * S->nlab);
    memset(Dl, 0, sizeof(double) * S->nlab);
    if (Hll) memset(Hll, 0, sizeof(double) * S->nlab * S->nlab);
    Nl[0] = S->norm0;
    Dl[0] = S->e0 * S->norm0;
    double pp = S->c[0] * S->c[0] * S->norm0, php = 0.0;
    double *dla = calloc((size_t)(u + S->nref), sizeof(double));
    double *pha = calloc((size_t)(u + S->nref), sizeof(double));
    for (int64_t i = 0; i < u; i++) {
        int64_t l = det_label(S, &buf[i].d, NULL, NULL);
        Nl[l] += buf[i].v * buf[i].v;
        pp += S->c[l] * S->c[l] * buf[i].v * buf[i].v;
    }
    /* 2. <v_l|H_D|v_l> and <psi_s|H|psi_s> over pairs (m, m') H-connected; the determinants are
     * visited label by label, so that one thread owns a row of Hll (no shared writes) */
    int64_t ntot = u + S->nref;
    int64_t *lstart = calloc((size_t)(S->nlab + 1), sizeof(int64_t));
    int64_t *lord = malloc(sizeof(int64_t) * (size_t)(ntot ? ntot : 1));
    for (int64_t x = 0; x < ntot; x++) {
        int64_t l = x < S->nref ? 0 : det_label(S, &buf[x - S->nref].d, NULL, NULL);
        lstart[l + 1]++;
    }
    for (int64_t l = 0; l < S->nlab; l++) lstart[l + 1] += lstart[l];
    {
        int64_t *fill = malloc(sizeof(int64_t) * (size_t)(S->nlab + 1));
        memcpy(fill, lstart, sizeof(int64_t) * (size_t)(S->nlab + 1));
        for (int64_t x = 0; x < ntot; x++) {
            int64_t l = x < S->nref ? 0 : det_label(S, &buf[x - S->nref].d, NULL, NULL);
            lord[fill[l]++] = x;
        }
        free(fill);
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t lgrp = 0; lgrp < S->nlab; lgrp++)
    for (int64_t q = lstart[lgrp]; q < lstart[lgrp + 1]; q++) {
        const int64_t i = lord[q] - S->nref;
        det_t d;
        double vi, ci;
        int64_t li;
        if (i < 0) { d = S->ref[i + S->nref]; vi = S->refc[i + S->nref]; li = 0; ci = S->c[0]; }
        else { d = buf[i].d; vi = buf[i].v; li = det_label(S, &d, NULL, NULL); ci = S->c[li]; }
        double dl = 0.0, ph = 0.0;
        if (li > 0) dl += hd_diag(S, &d) * vi * vi;
        ph += ci * vi * h_diag(S, &d) * ci * vi;
        if (Hll) Hll[li * S->nlab + li] += vi * h_diag(S, &d) * vi;
        int occl[2 * MAXN], empl[2 * MAXN], no = 0, ne = 0;
        for (int so = 0; so < 2 * n; so++) { if (occ(&d, so, n)) occl[no++] = so; else empl[ne++] = so; }
        for (int kind = 1; kind <= 2; kind++)
            for (int x1 = 0; x1 < no; x1++)
                for (int x2 = (kind == 1 ? x1 : x1 + 1); x2 < (kind == 1 ? x1 + 1 : no); x2++)
                    for (int y1 = 0; y1 < ne; y1++)
                        for (int y2 = (kind == 1 ? y1 : y1 + 1); y2 < (kind == 1 ? y1 + 1 : ne); y2++) {
                            det_t m = d;
                            clrb(&m, occl[x1], n); setb(&m, empl[y1], n);
                            if (kind == 2) { clrb(&m, occl[x2], n); setb(&m, empl[y2], n); }
                            int64_t lm = det_label(S, &m, NULL, NULL);
                            if (lm < 0) continue;
                            double vm;
                            if (lm == 0) vm = phi0(S, &m);
                            else { int64_t j = find_dv(buf, u, &m); vm = j >= 0 ? buf[j].v : 0.0; }
                            if (vm == 0.0) continue;
                            ph += ci * vi * h_elem(S, &d, &m) * S->c[lm] * vm;
                            if (Hll) Hll[li * S->nlab + lm] += vi * h_elem(S, &d, &m) * vm;
                            if (li > 0 && lm == li) dl += vi * hd_elem(S, &d, &m) * vm;
                        }
        dla[i + S->nref] = dl;
        pha[i + S->nref] = ph;
    }
    for (int64_t i = -S->nref; i < u; i++) {
        php += pha[i + S->nref];
        if (i >= 0) Dl[det_label(S, &buf[i].d, NULL, NULL)] += dla[i + S->nref];
    }
    out[0] = pp; out[1] = php; out[2] = (double)u;
    free(buf); free(dla); free(pha); free(lstart); free(lord);
    return 0;
}
