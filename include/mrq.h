/*
 * mrq.h - C ABI of the GB300 (sm_103a) local-estimator library for stochastic strongly
 * contracted SC-NEVPT2(s) and SC-MRCI(s) (Mahajan, Blunt, Sabzevari, Sharma,
 * arXiv:1909.06935).
 *
 * The library owns one CUDA context slot per `mrq_ctx` and keeps everything the walk needs
 * resident in device memory: integrals, the reference hash table, sampling coefficients,
 * walker states and accumulators.  All arithmetic is FP64.
 *
 * Conventions shared by every call:
 *  - n = n_core + n_act + n_virt spatial orbitals (n <= 128), ordered core, active, virtual;
 *    n_core <= 64, n_act <= 32.  A walker's block keeps one reach-back candidate list per warp in
 *    shared memory: systems whose lists are too long for eight warps run with four, two or one
 *    (mrq_load_hamiltonian returns MRQ_TOO_LARGE only when one warp's list does not fit).
 *  - A determinant is 2W uint64 words, W = ceil(n/64): alpha occupation bits (bit p of word
 *    p/64 set when spatial orbital p holds an alpha electron), then beta.  Its sign convention
 *    is |det> = prod_{alpha p ascending} a+_p prod_{beta p ascending} a+_p |vac>.
 *  - Integrals are chemists' (pq|rs), 8-fold packed: eri[P(P(p,q),P(r,s))],
 *    P(x,y) = x(x+1)/2 + y for x >= y, so eri has P(P+1)/2 entries with P = n(n+1)/2.
 *  - The perturber label of a determinant (the subspace S_l^(k) of Sec. II A, read in spin
 *    orbitals) is its set H of empty core spin orbitals and its set P of occupied virtual spin
 *    orbitals, |H| <= 2, |P| <= 2: label = rank(H) * nP + rank(P), rank(empty) = 0,
 *    rank({x}) = 1 + x, rank({x<y}) = 1 + m + y(y-1)/2 + x, where core spin orbital x =
 *    sigma*n_core + i, virtual spin orbital x = sigma*n_virt + a, m = number of spin orbitals
 *    of that space, nP = 1 + 2 n_virt + C(2 n_virt, 2).  Label 0 is the CAS.  The number of
 *    labels is nH * nP, nH = 1 + 2 n_core + C(2 n_core, 2).
 *  - Its type is 3h + p (h = |H|, p = |P|): 0 CAS, 1 S_r, 2 S_rs, 3 S_i, 4 S_i,r, 5 S_i,rs,
 *    6 S_ij, 7 S_ij,r, 8 S_ij,rs (NEVPT notation of Angeli et al.).
 *  - Pointer arguments may address host or device memory (unified addressing decides);
 *    the library copies inputs in before returning, so the caller keeps ownership.
 *  - Every call returns 0 or a negative `mrq_status`; `mrq_last_error` gives the message.
 *    A context must be used by one host thread at a time.
 */
#ifndef MRQ_H
#define MRQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mrq_ctx mrq_ctx;

enum mrq_status {
    MRQ_OK = 0,
    MRQ_INVALID_ARG = -1,
    MRQ_NOT_LOADED = -2,
    MRQ_BAD_REFERENCE = -3,   /* a determinant with a core hole, a virtual electron, the wrong
                                 electron count, or a duplicate */
    MRQ_OOM = -4,
    MRQ_HASH_OVERFLOW = -5,   /* a hash probe ran past its bound */
    MRQ_DEVICE_TIMEOUT = -6,
    MRQ_CUDA_ERROR = -7,
    MRQ_NO_MOVE = -8,         /* a walker found no determinant to move to (all rates zero) */
    MRQ_TOO_LARGE = -9
};

enum mrq_method { MRQ_SC_NEVPT2 = 0, MRQ_SC_MRCI = 1 };

#define MRQ_NTYPES 9

/* Sampling parameters. */
typedef struct {
    int64_t n_walkers;      /* independent continuous-time walkers (Sec. II B) */
    int64_t n_steps;        /* steps per walker in this call (including burn-in on a fresh start) */
    int64_t burn_in;        /* leading steps of every walker left out of the averages */
    uint64_t seed;          /* Philox4x32-10 key of the move selection */
    int32_t n_groups;       /* G walker groups for jackknife errors (walker w is in group w mod G) */
    int32_t method;         /* mrq_method: informative; both estimators are always accumulated */
    double screen_tau;      /* perturbers with N_l/N_0 below this are screened out (Sec. II C) */
    int32_t warps_per_walker;  /* 1, 2, 4 or 8 warps in each walker's thread block (at most what the
                                  system's candidate lists allow); 0 keeps the context's setting (by
                                  default chosen from the system's size, see mrq_set_launch) */
    int32_t steps_per_check;   /* mrq_sample with target_sigma: steps between error checks (0: n_steps/16) */
    double target_sigma;    /* mrq_sample stops early once the jackknife sigma of E^(2) (method
                               SC_NEVPT2) or of E (SC_MRCI) is at or below this; 0 = off */
} mrq_sample_params;

/* Result of a sampling run (all energies in Hartree). */
typedef struct {
    double e0;                      /* <phi0|H|phi0>/<phi0|phi0> */
    double e2, e2_sigma;            /* SC-NEVPT2 second-order energy (Eq. 15), jackknife sigma */
    double e_var, e_var_sigma;      /* <E_L> of the sampled function (Eq. 4): SC-MRCI energy for given c */
    double a0sq, a0sq_sigma;        /* c_0^2 <phi0|phi0>/<psi|psi> (Eq. 11-12) */
    double e_mrci_q;                /* e_var + (1 - a0sq)(e_var - e0), Davidson +Q (Eq. 10) */
    double type_norm[MRQ_NTYPES], type_norm_sigma[MRQ_NTYPES];  /* sum of kept N_l/N_0 per type */
    double type_e2[MRQ_NTYPES], type_e2_sigma[MRQ_NTYPES];      /* E^(2) contribution per type */
    double type_screened[MRQ_NTYPES];     /* visited labels screened out, per type */
    double screened_norm;                 /* sum of N_l/N_0 over screened labels */
    double n_labels_visited;
    int64_t type_steps[MRQ_NTYPES];       /* walker steps spent at each type (class mix) */
    int64_t walker_steps;                 /* accumulated (post burn-in) walker steps */
    int64_t total_steps;                  /* all walker steps taken by this context */
    double seconds;                       /* device time of the walk kernels since mrq_walkers_init */
    int64_t walk_launches;                /* walk kernel launches since mrq_walkers_init */
    int32_t status;
    int32_t reserved;
} mrq_result;

/* Per-determinant local quantities (debug / parity; Eq. 5, Eq. 16). */
typedef struct {
    double S;         /* sum_m Gamma_nm, Gamma_nm = |H_nm psi_s(m)/psi_s(n)| */
    double e_local;   /* E_L(n) = sum_m H_nm psi_s(m)/psi_s(n) including m = n (Eq. 5) */
    double num;       /* sum_m (H_D)_nm psi_s(m)/psi_s(n) over m of n's label (Eq. 16), 0 in the CAS */
    double h_nn, hd_nn, psi;   /* <n|H|n>, <n|H_D|n>, psi_s(n) */
    int64_t label;    /* -1 outside CAS and FOIS */
    int64_t type;
    int64_t n_neighbours;
    int64_t n_candidates; /* reach-back candidates tried (hash lookups of neighbours and of their CAS images) */
    int64_t n_probes;     /* hash slots read (16 B each) */
    int64_t n_gathers;    /* 8 B random reads of integrals and per-orbital / per-label tables */
    int64_t n_terms;      /* products <m|H|k> phi0(k) summed into the overlaps O(m) (one FP64 FMA each) */
} mrq_local;

/* Per-neighbour record of mrq_debug_local. */
typedef struct {
    uint64_t det[4];  /* first 2W words used */
    double h, hd;     /* <n|H|m>, <n|H_D|m> (0 unless same label and n outside the CAS) */
    double o;         /* phi0(m) for a CAS m, O(m) = <m|H|phi0> otherwise (Eq. 6-7) */
    double psi;       /* psi_s(m) */
    double gamma;     /* |H_nm psi_s(m)/psi_s(n)| */
    uint32_t exc;     /* removed spin orbitals r1<=r2, added a1<=a2: r1 | r2<<8 | a1<<16 | a2<<24 */
    uint32_t pad;
} mrq_neighbour;

/* Create a context on CUDA device `device`.  Returns 0 or a negative status. */
int mrq_create(mrq_ctx** out, int device);

/* Free everything the context holds (device memory, stream, events).  NULL is ignored. */
void mrq_destroy(mrq_ctx* ctx);

/* Message of the last failing call on this context ("" when none). Valid until the next call. */
const char* mrq_last_error(const mrq_ctx* ctx);

/* Use `stream` (a cudaStream_t, or NULL for the context's own stream) for all later work. */
int mrq_set_stream(mrq_ctx* ctx, void* stream);

/*
 * Load the Hamiltonian (the problem statement of Sec. II A and the Dyall partition of
 * Sec. II C): n_core doubly occupied core, n_act active and n_virt virtual spatial orbitals,
 * n_alpha/n_beta electrons in total, h1 (n*n row-major, symmetric), eri (8-fold packed, see
 * above) and a constant e_core added to every diagonal element (e.g. nuclear repulsion).
 * Replaces any previous Hamiltonian and invalidates the reference and walkers.
 * Errors: MRQ_INVALID_ARG (sizes), MRQ_OOM, MRQ_CUDA_ERROR.
 */
int mrq_load_hamiltonian(mrq_ctx* ctx, int n_core, int n_act, int n_virt, int n_alpha, int n_beta,
                         const double* h1, const double* eri, double e_core);

/*
 * Load the reference phi0 (Sec. II D: a selected-CI vector kept in a hash table): n_det
 * determinants (n_det x 2W words) with coefficients (need not be normalised).  Builds the
 * device hash table and the one-time quantities of Sec. II C: E0 = <phi0|H|phi0>/<phi0|phi0>,
 * the active 1-RDM, the generalised-Fock diagonal eps, and the core-averaged operators.
 * Also sets the sampling coefficients to c_0 = 1, c_l = 0.1 for every label (override with
 * mrq_set_coeffs).  Errors: MRQ_NOT_LOADED (no Hamiltonian), MRQ_BAD_REFERENCE,
 * MRQ_HASH_OVERFLOW, MRQ_OOM, MRQ_CUDA_ERROR.
 */
int mrq_load_reference(mrq_ctx* ctx, int64_t n_det, const uint64_t* dets, const double* coeffs);

/*
 * Coefficients c_l of the sampled function psi = c_0 phi0 + sum_l c_l psi_l (Eq. 17 for
 * SC-NEVPT2(s), the SC-MRCI(s) wave function of Sec. II B for given c), one per label in
 * label order (see above); n_labels must equal nH * nP.  Errors: MRQ_INVALID_ARG, MRQ_NOT_LOADED.
 */
int mrq_set_coeffs(mrq_ctx* ctx, int64_t n_labels, const double* c);

/* Number of labels nH * nP of the loaded Hamiltonian (0 when none). */
int64_t mrq_n_labels(const mrq_ctx* ctx);

/*
 * Setup quantities after mrq_load_reference: out[0] = E0, out[1] = <phi0|phi0>, out[2] = E_core
 * (core energy), out[3] = sum of core eps, out[4] = index (input order) of the largest |c|
 * determinant (the walkers' start).  eps receives n doubles (or NULL), gamma n_act^2 (or NULL).
 */
int mrq_setup_info(mrq_ctx* ctx, double* out5, double* eps, double* gamma);

/*
 * Local quantities of n determinants (Eq. 5, Eq. 16, Sec. II D), for parity checks: local[i]
 * for det i; when nb != NULL the neighbours of det i go to nb[i*max_nb ...] (at most max_nb
 * each, in the library's enumeration order; local[i].n_neighbours gives the full count).
 */
int mrq_debug_local(mrq_ctx* ctx, int64_t n, const uint64_t* dets, mrq_local* local,
                    int64_t max_nb, mrq_neighbour* nb);

/*
 * Start n_walkers fresh walkers at the largest-|phi0| determinant and clear the accumulators
 * (G = n_groups groups).  Errors: MRQ_NOT_LOADED, MRQ_INVALID_ARG, MRQ_OOM.
 */
int mrq_walkers_init(mrq_ctx* ctx, const mrq_sample_params* p);

/*
 * Advance every walker by n_steps continuous-time steps (Sec. II B; first-reaction form of
 * Gillespie's algorithm with Philox4x32-10 clocks keyed on (seed; exc, step, walker)),
 * accumulating the estimators of Eq. 4, 12 and 16 after each walker's burn-in.  Asynchronous
 * on the context stream.  Errors: MRQ_NOT_LOADED, MRQ_CUDA_ERROR.
 */
int mrq_walkers_advance(mrq_ctx* ctx, int64_t n_steps);

/*
 * Finalize the accumulators into `out` (Eq. 14-15 with screening at screen_tau, jackknife
 * errors over the G groups).  Synchronises the stream; reports device-side error flags
 * (MRQ_HASH_OVERFLOW, MRQ_NO_MOVE) in the return value and out->status.
 */
int mrq_finalize(mrq_ctx* ctx, mrq_result* out);

/*
 * Same result as mrq_finalize, but the call allocates no device memory: its partial sums go to
 * a fixed array compiled into the library (MRQ_NOALLOC_SCRATCH_DOUBLES doubles, 4 MiB), which
 * every GPU that loads the library keeps until the process exits.  For callers that must not
 * call cudaMalloc/cudaFree while they run, e.g. a serving loop whose device memory is all
 * handed to its own pool allocator, or a latency-bound loop that cannot absorb the device
 * synchronisation an allocation may cause.  The paper has no counterpart; it is an
 * implementation convenience.  The array's device address is looked up in mrq_create, once
 * per device.  Needs (n_groups + 1) * ceil(n_labels / 8192) * 45 doubles of scratch and
 * returns MRQ_TOO_LARGE when that exceeds the fixed size.  All calls on one device share the
 * array (each call overwrites what it uses), so calls whose GPU work overlaps race: issue them
 * on one stream, or wait for one to finish before the next.
 */
#define MRQ_NOALLOC_SCRATCH_DOUBLES (1 << 19)
int mrq_finalize_noalloc(mrq_ctx* ctx, mrq_result* out);

/*
 * Batched walk: advance the walkers of n contexts (independent systems, each initialised with
 * mrq_walkers_init) by n_steps in one walk launch per determinant width and occupancy class (the
 * walk blocks per SM a system's shared memory allows, so that small systems are not held to the
 * occupancy of the largest), so that many small systems fill the GPU together (the paper runs each
 * system on its own; walkers are independent Markov chains, Sec. II B).  Walker ids, seeds and accumulators stay per context, so every
 * trajectory is the same as when its context advances alone.  All contexts must be on one device;
 * the launch uses ctxs[0]'s stream after waiting for every context's stream, and returns after it
 * completes.  The walk time is reported by mrq_finalize on ctxs[0] only.
 * Errors: MRQ_INVALID_ARG (null / duplicate contexts, different devices), MRQ_NOT_LOADED.
 */
int mrq_batch_advance(mrq_ctx* const* ctxs, int n, int64_t n_steps);

/*
 * Launch configuration of a context's walks (no counterpart in the paper: a GPU scheduling
 * choice that leaves every trajectory and accumulator the same, up to the order of the FP64
 * additions).  warps_per_walker in {1, 2, 4, 8}: the warps of the thread block that takes one walker's
 * step (they split its neighbours into interleaved work units); 0, the default, chooses from the
 * system's work units per CAS walker (8 for 512 or more, 4 for 128 or more, else 2; a batch takes
 * the largest of its systems' choices);
 * steps_per_launch >= 1 splits an advance into launches of that many steps, each re-ordering the
 * walker slots first (0, the default: one launch per advance); use_graph != 0 makes
 * mrq_batch_advance, with ctxs[0] this context, capture one launch of steps_per_launch steps (the
 * reporting interval: slot sort + walk) into a CUDA graph once per batch layout and replay it.
 * Errors: MRQ_INVALID_ARG.
 */
int mrq_set_launch(mrq_ctx* ctx, int warps_per_walker, int steps_per_launch, int use_graph);

#define MRQ_TUNE_MAX 16
typedef struct {
    int warps_per_walker;     /* the fastest configuration, now set on every context of the batch */
    int steps_per_launch;
    int n_tried;
    int tried_warps_per_walker[MRQ_TUNE_MAX];
    int tried_steps_per_launch[MRQ_TUNE_MAX];
    double tried_ms[MRQ_TUNE_MAX];   /* device time of trial_steps steps, best of up to 3 */
} mrq_tune_result;

/*
 * Autotuner of the batched walk: times trial_steps (1..1024) steps of the batch for every
 * warps_per_walker in {2, 4, 8} and steps_per_launch in {1, 4, 16} (those <= trial_steps), on a
 * scratch copy of the walkers with accumulation off, so the contexts' walkers and accumulators
 * are left as they were; then sets the fastest pair on every context (mrq_set_launch, keeping
 * use_graph).  out may be NULL.  Errors: as mrq_batch_advance, MRQ_INVALID_ARG for trial_steps.
 */
int mrq_tune_batch(mrq_ctx* const* ctxs, int n, int64_t trial_steps, mrq_tune_result* out);

/* mrq_walkers_init for each context (params[i]), mrq_batch_advance(params[0].n_steps), and
 * mrq_finalize of each into out[i].  Every params[i].n_steps must be equal. */
int mrq_sample_batch(mrq_ctx* const* ctxs, int n, const mrq_sample_params* params, mrq_result* out);

/* ------------------------------------------------------------------------------------------
 * Request server (serving form; the paper has no counterpart - it runs one system per job).
 * Sampling requests for different systems wait in a FIFO queue; each scheduling round admits
 * queued requests while the device-memory budget and the active-slot limit allow, advances all
 * active requests together (mrq_batch_advance), finalizes them and retires those that reached
 * their target sigma of E^(2) or their step limit.  A request's walkers take the same steps
 * whatever else is active, so its trajectory is the same alone and in the mix.
 * ------------------------------------------------------------------------------------------ */
typedef struct mrq_server mrq_server;

enum mrq_request_state { MRQ_REQ_QUEUED = 0, MRQ_REQ_RUNNING = 1, MRQ_REQ_DONE = 2, MRQ_REQ_FAILED = 3,
                         MRQ_REQ_CANCELLED = 4 };

typedef struct {
    int32_t device;
    int32_t max_active;          /* requests resident at once */
    int64_t hbm_budget_bytes;    /* device bytes the resident requests may use (estimated per request) */
    int64_t steps_per_round;     /* walker steps per batched launch */
} mrq_server_params;

typedef struct {
    int32_t n_core, n_act, n_virt, n_alpha, n_beta, reserved;
    double e_core;
    const double* h1;            /* as mrq_load_hamiltonian */
    const double* eri;
    int64_t n_det;               /* as mrq_load_reference */
    const uint64_t* dets;
    const double* coeffs;
    int64_t n_labels;            /* 0: default coefficients; else as mrq_set_coeffs */
    const double* c;
    mrq_sample_params params;    /* n_walkers, burn_in, seed, n_groups, screen_tau (n_steps unused) */
    double target_sigma;         /* stop when the jackknife sigma of E^(2) is at most this (0: never) */
    int64_t max_steps;           /* stop after this many steps per walker */
} mrq_request;

typedef struct {
    int32_t state;               /* mrq_request_state */
    int32_t status;              /* mrq_status of a failed request */
    int64_t steps_done;          /* steps per walker so far */
    double queue_seconds;        /* submit -> admission */
    double total_seconds;        /* submit -> done (or now) */
    mrq_result result;           /* latest finalize (after every round while running) */
} mrq_request_status;

/* Create a server; nothing is loaded until requests are admitted. */
int mrq_server_create(mrq_server** out, const mrq_server_params* p);
/* Queue a request; the inputs are copied (the caller keeps ownership).  A request whose estimated
 * footprint exceeds the whole budget is recorded as failed with MRQ_TOO_LARGE. */
int mrq_server_submit(mrq_server* s, const mrq_request* req, int64_t* ticket);
/* State, timings and latest result of a ticket. */
int mrq_server_poll(mrq_server* s, int64_t ticket, mrq_request_status* out);
/* Cancel a queued request at once, a running one at the end of the current round. */
int mrq_server_cancel(mrq_server* s, int64_t ticket);
/* Run one scheduling round on the calling thread (not while the background loop runs). */
int mrq_server_step(mrq_server* s);
/* Start / stop a background thread that runs rounds while there is work. */
int mrq_server_start(mrq_server* s);
int mrq_server_stop(mrq_server* s);
/* out4 = queued, active, estimated resident bytes, walker steps advanced so far. */
int mrq_server_info(mrq_server* s, int64_t* out4);
const char* mrq_server_last_error(const mrq_server* s);
/* Stop, free every resident request, destroy. */
void mrq_server_destroy(mrq_server* s);

/* mrq_walkers_init + mrq_walkers_advance(p->n_steps) + mrq_finalize.  With p->target_sigma > 0
 * the walk advances steps_per_check steps at a time and stops at the first check (after the
 * burn-in) whose sigma is at or below the target, or after n_steps; out->total_steps says how far
 * it went.  Errors: as the three calls. */
int mrq_sample(mrq_ctx* ctx, const mrq_sample_params* p, mrq_result* out);

/*
 * Raw accumulators of the last walk: accN/accU (G x n_labels), accW/accE (G), type_steps (9).
 * Any pointer may be NULL.  Synchronises the stream.
 */
int mrq_read_accumulators(mrq_ctx* ctx, double* accN, double* accU, double* accW, double* accE,
                          int64_t* type_steps);

/*
 * SC-MRCI(s) energy gradient of the last walk (Eq. 8-9, Sec. II B): for the sampled function
 * psi = sum_l c_l psi_l, <n|d psi/d c_l> / <n|psi> = delta_{l,l_n} / c_l, so
 *   grad[l] = < delta_{l,l_n} / c_l (E_L(n) - E) >,  E = <E_L>,
 * averaged with the walk's residence weights over all groups.  Like Eq. 8 it leaves out the
 * factor 2 of the derivative of <psi|H|psi>/<psi|psi> for a real psi.  grad receives n_labels
 * doubles (host or device memory, or NULL), energy the estimate E (or NULL).
 * Errors: MRQ_NOT_LOADED (no walk since the reference was loaded).
 */
int mrq_mrci_gradient(mrq_ctx* ctx, double* grad, double* energy);

/*
 * One AMSGrad step (Reddi, Kale, Kumar, ICLR 2018, without bias correction; the optimiser of
 * Sec. II B) on the context's coefficients c_l, l >= 1, with the gradient of the last
 * mrq_mrci_gradient call:  m = b1 m + (1-b1) g,  v = b2 v + (1-b2) g^2,  vhat = max(vhat, v),
 * c -= lr m / (sqrt(vhat) + eps).  c_0 stays fixed: the energy does not depend on the scale of c.
 * m, v, vhat live on the device, start at zero and are reset by mrq_set_coeffs.
 * Errors: MRQ_NOT_LOADED (no gradient yet), MRQ_INVALID_ARG (lr <= 0, beta outside [0,1), eps <= 0).
 */
int mrq_amsgrad_step(mrq_ctx* ctx, double lr, double beta1, double beta2, double eps);

/* Current sampling coefficients c_l of Eq. 17 (after any AMSGrad steps): n_labels doubles into c
 * (host or device memory, owned by the caller).  Errors: MRQ_INVALID_ARG (null), MRQ_NOT_LOADED. */
int mrq_read_coeffs(mrq_ctx* ctx, double* c);

/* Raw gradient sums of the last walk per walker group (Eq. 8-9 with residence weights w = 1/S),
 * n_groups x n_labels doubles each, row-major by group (host memory owned by the caller; either
 * may be NULL): accA[g][l] = sum w E_L / c_l, accB[g][l] = sum w / c_l.  n_groups is the last
 * mrq_walkers_init's.  Errors: MRQ_NOT_LOADED (no walk yet). */
int mrq_read_gradient_sums(mrq_ctx* ctx, double* accA, double* accB);

/* Walker determinants (n_walkers x 2W words) and psi_s values; either may be NULL. */
int mrq_read_walkers(mrq_ctx* ctx, uint64_t* dets, double* psi);

/*
 * The move race's screen, for parity tests (Sec. II B: the rejection-free continuous-time walk,
 * taken in the first-reaction form of Gillespie's algorithm; each neighbour m draws the clock
 * t = -ln(u)/Gamma_nm and the smallest t wins).  The walk evaluates the exact FP64 clock only for
 * candidates that pass an FP32 screen against the best clock so far.  For i < n: u = (k53[i] + 1)
 * 2^-53 with k53[i] < 2^53 (the 53 random bits of the walk's Philox4x32-10 draw), exact[i] =
 * -ln(u)/rate[i] in FP64, and pass[i] = 1 when the screen lets a candidate of rate rate[i] through
 * against the best clock t_best[i] (infinity: none yet), formed exactly as the walk forms it.  The
 * screen never rejects a candidate whose exact clock is below t_best[i].  All arrays are n long,
 * host or device memory owned by the caller.  Errors: MRQ_INVALID_ARG (null pointers, n <= 0, a
 * k53 with more than 53 bits), MRQ_CUDA_ERROR.
 */
int mrq_debug_race_screen(mrq_ctx* ctx, int64_t n, const uint64_t* k53, const double* rate, const double* t_best,
                          uint8_t* pass, double* exact);

/*
 * Persisting-L2 window of this context's walk launches (no counterpart in the paper; a GB300
 * cache setting).  With fraction > 0 every walk launch marks the physicists' integral tables (the
 * entries every reach-back term reads) as persisting in L2, with a hit ratio that fits them into
 * fraction x the device's maximum persisting carve-out, which this call's launches set as the
 * CUDA context's persisting-L2 limit (a per-process limit that ends with the context; no device
 * setting outlasts the process).  0 (the default) launches without a window.  Batched launches
 * (several systems) never take one.  Errors: MRQ_INVALID_ARG (fraction outside [0, 1]).
 */
int mrq_set_l2_window(mrq_ctx* ctx, double fraction);

/*
 * Deadline of this context's host waits (failure detection; the paper has no counterpart).
 * With seconds > 0, every call that waits for the device (mrq_finalize, mrq_finalize_noalloc,
 * mrq_sample, the readers, and the wait for earlier work at the start of a load) gives up after
 * that long and returns MRQ_DEVICE_TIMEOUT; nothing is written to its outputs, the device work
 * keeps running, and the next call waits for it again.  Set-up calls apply the deadline only to
 * the wait for earlier work, never to their own kernels.  0 (the default) waits without limit.
 * Errors: MRQ_INVALID_ARG (negative).
 */
int mrq_set_deadline(mrq_ctx* ctx, double seconds);

/*
 * Lower the walk's device-side bounds, so that tests can make them run out (failure detection;
 * the paper has no counterpart).  max_probe (1..64) bounds the hash slots a lookup reads (the
 * table itself allows 64); cand_cap bounds the entries of one candidate list of the grouped
 * CAS-walker path (at most what the loaded system needs).  A lookup or list that runs past its
 * bound sets a device flag and the next finalize returns MRQ_HASH_OVERFLOW or MRQ_TOO_LARGE; the
 * walk itself always ends (the overflowing lookup reads as absent, the list is cut).  0 restores
 * the default of either.  A bound lowered before mrq_load_reference also bounds the table's
 * insertions.  Errors: MRQ_INVALID_ARG.
 */
int mrq_debug_set_limits(mrq_ctx* ctx, int max_probe, int cand_cap);

/*
 * Measured ceilings of the device for the walk's roofline (the paper has no counterpart): the walk
 * is FP64 arithmetic on randomly gathered table entries.  out3[0] = FP64 FMA rate (flop/s) of
 * independent register FMA chains on every SM; out3[1] = random 8-byte reads per second from a
 * 16 MiB table (resident in L2); out3[2] = the same from a 4 GiB table (HBM).  Allocates and frees
 * 4 GiB on `device`, runs for about a tenth of a second.  Errors: MRQ_INVALID_ARG, MRQ_CUDA_ERROR.
 */
int mrq_probe_peaks(int device, double* out3);

/*
 * Replace this context's accumulators by given per-group sums, e.g. the union of the groups of
 * several independent walks: the combining step of a run whose ranks each walk their own walkers
 * (the paper's implementation reduces over MPI ranks of walkers, Sec. III).  A rank reads its
 * sums with mrq_read_accumulators / mrq_read_gradient_sums; rank 0 concatenates every rank's
 * groups (rank r's group g becomes group r G + g) and loads them here, and mrq_finalize then
 * reports the combined estimates with jackknife errors over all n_groups groups.  accN, accU,
 * accA, accB: n_groups x n_labels row-major (accA, accB may be NULL: zero); accW, accE: n_groups;
 * type_steps: MRQ_NTYPES counts; total_steps: walker steps of all the walks.  Host or device
 * memory, copied in.  The context's walkers are left out of step (mrq_walkers_init starts a new
 * walk).  Errors: MRQ_NOT_LOADED (no reference), MRQ_INVALID_ARG (1 <= n_groups <= 64), MRQ_OOM.
 */
int mrq_load_accumulators(mrq_ctx* ctx, int32_t n_groups, const double* accN, const double* accU, const double* accW,
                          const double* accE, const double* accA, const double* accB, const int64_t* type_steps,
                          int64_t total_steps);

/*
 * Heat-bath cutoff of the walk (Sec. II D generates the excitations by the heat-bath algorithm,
 * whose cutoff the paper sets to zero: all excitations).  With eps > 0 every double excitation
 * whose matrix element |<ab||ij>| (|<ab|ij>| for opposite spins) is below eps is dropped wherever
 * the walk uses one: the walker's neighbours (E_L, rates, moves), the reach-back overlaps O(m),
 * and the H_D numerator; singles and diagonals stay exact, and E0 is the unscreened <phi0|H|phi0>.
 * The result is the method applied to that screened Hamiltonian (an approximation; eps = 0
 * restores the exact method).  Reloading the Hamiltonian resets it to 0.  Errors: MRQ_NOT_LOADED,
 * MRQ_INVALID_ARG (negative or not finite).
 */
int mrq_set_heat_bath_cutoff(mrq_ctx* ctx, double eps);

/*
 * Copy the loaded integrals back (h1: n*n doubles, eri: the 8-fold packed array; either may be
 * NULL), e.g. the semicanonical core and virtual orbitals Dyall's H_D assumes (Sec. II C) after
 * mrq_sci_reference rotated them.  Errors: MRQ_NOT_LOADED, MRQ_CUDA_ERROR.
 */
int mrq_read_hamiltonian(mrq_ctx* ctx, double* h1, double* eri);

/* Parameters of mrq_sci_reference. */
typedef struct {
    int32_t n_strings;      /* selected occupation strings per spin; the reference holds n_strings^2
                               determinants (clamped to the string space; at most 4096) */
    int32_t n_seed_strings; /* strings of lowest one-spin energy whose product space seeds the
                               selection (clamped to the string space; at most n_strings) */
    double tol;             /* Davidson residual-norm bound of both solves (> 0) */
    int32_t max_iter;       /* Davidson iterations per solve (>= 1) */
    int32_t max_sub;        /* Davidson subspace size before a restart (2..64) */
    int32_t semicanonical;  /* 1: rotate the core and virtual orbitals so that the generalised Fock
                               blocks F_cc and F_vv are diagonal, and reload the Hamiltonian */
    int32_t reserved;
} mrq_sci_params;

/* What mrq_sci_reference built. */
typedef struct {
    double energy;          /* variational energy of phi0 in the selected product space (E_core and
                               e_core included) */
    double seed_energy;     /* lowest energy in the seed product space */
    double residual;        /* Davidson residual norm of phi0 */
    double fock_offdiag;    /* largest |F_pq|, p != q, inside the core and virtual blocks before the
                               rotation (0 when semicanonical = 0) */
    double seconds;         /* wall time of the call */
    int64_t n_det;          /* determinants loaded as the reference (n_strings^2) */
    int32_t n_strings, n_seed_strings;   /* as used */
    int32_t iters_seed, iters;           /* Davidson iterations of the seed and the final solve */
} mrq_sci_result;

/*
 * Build the reference phi0 on the device as a heat-bath selected CI of the active space (the
 * selected-CI reference of Sec. II D; Sz = 0, so n_alpha must equal n_beta) and load it as
 * mrq_load_reference would.  The Hamiltonian in the active space is the core-averaged one:
 * E_core + sum_tu h_tu E_tu + 1/2 sum (tu|vw)(E_tu E_vw - delta_uv E_tw), h = h1 + sum_i [2(tu|ii) -
 * (ti|iu)].  Steps: the n_seed_strings strings of lowest one-spin energy (first on ties) span a seed
 * product space, whose lowest eigenvector C0 (Davidson) weighs each seed string s by w_s =
 * (sum_b C0[s,b]^2 + sum_a C0[a,s]^2)/2; every string s' scores max_s |<s'|H1|s>| sqrt(w_s) (H1 the
 * one-spin part of the Hamiltonian; seeds score infinity); the n_strings best (first on ties) span
 * the final product space, solved again from the embedded C0.  The sign makes the largest |c|
 * positive.  Determinant k = a n_strings + b holds alpha string a and beta string b of the
 * selection (strings in lexicographic order of their sorted orbital lists; bit t = active orbital
 * t).  With semicanonical = 1 the generalised Fock matrix F_pq = h_pq + sum_i [2(pq|ii) - (pi|iq)] +
 * sum_tu gamma_tu [(pq|tu) - (pt|uq)/2] of the new reference (gamma its spin-summed active 1-RDM)
 * is diagonalised in the core and virtual blocks (eigenvalues ascending), h1 and (pq|rs) are
 * rotated on the device and reloaded (as mrq_load_hamiltonian would; mrq_read_hamiltonian returns
 * them); the active orbitals, and so phi0, are unchanged.  strings_out (n_strings uint32, or NULL)
 * receives the selected strings, coeffs_out (n_strings^2 doubles, or NULL) the coefficients.  The
 * one-spin string space C(n_act, n_alpha - n_core) is limited to 65,536 strings.  Errors:
 * MRQ_NOT_LOADED, MRQ_INVALID_ARG, MRQ_TOO_LARGE, MRQ_OOM, MRQ_CUDA_ERROR, and those of the loads.
 */
int mrq_sci_reference(mrq_ctx* ctx, const mrq_sci_params* p, mrq_sci_result* out, uint32_t* strings_out,
                      double* coeffs_out);

#ifdef __cplusplus
}
#endif

#endif /* MRQ_H */
