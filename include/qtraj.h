/*
 * qtraj.h -- C ABI of libqtraj, the GB300 (sm_103a) engine for the quantum-trajectory hot path of
 * QTraj 1.0 (Brambilla et al., arXiv:2107.06147): many independent waiting-time Monte-Carlo
 * wave-function trajectories of the heavy-quarkonium radial wave function u_l(r) under the
 * non-Hermitian OQS+pNRQCD Hamiltonian, and their overlaps with the vacuum Coulomb states.
 *
 * Conventions shared by every entry point:
 *   - every call returns a qtraj_status; nothing throws across the ABI; qtraj_last_error() gives
 *     a message for the last failing call on the calling thread;
 *   - GPU work is enqueued on the caller's stream (a cudaStream_t passed as void*, NULL = the legacy
 *     default stream) and is asynchronous unless the call says it synchronises;
 *   - the caller owns every buffer it passes and the library never frees caller memory; device
 *     buffers are plain device pointers with byte sizes; the library owns the context and its
 *     internal read-only tables (twiddles, phase tables, Coulomb basis), which it allocates in
 *     qtraj_create/qtraj_init and frees in qtraj_destroy;
 *   - one context is used by one host thread at a time; separate contexts are independent.
 *
 * Units: lengths in GeV^-1, energies and temperatures in GeV, proper time tau in fm/c
 * (hbar c = 0.1973269804 GeV fm converts the step dt to fm/c).
 */
#ifndef QTRAJ_H
#define QTRAJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qtraj_ctx qtraj_ctx;

typedef enum {
    QTRAJ_OK = 0,
    QTRAJ_EINVAL = 1,     /* bad argument: sizes, ranges, null pointers, unsupported N */
    QTRAJ_ENOMEM = 2,     /* workspace too small, or a host/device allocation failed */
    QTRAJ_ECUDA = 3,      /* a CUDA runtime call failed (message in qtraj_last_error) */
    QTRAJ_ETIMEOUT = 4,   /* a bounded device wait ran out */
    QTRAJ_ENONFINITE = 5, /* a trajectory norm became NaN/Inf (flag set in its record) */
    QTRAJ_EBUSY = 6       /* the context has queued work that this call would overwrite */
} qtraj_status;

/* arithmetic of the step: the norm, the waiting-time comparison and the overlaps are FP64 in all */
typedef enum { QTRAJ_FP64 = 0, QTRAJ_FP32 = 1 } qtraj_precision;

/* QTRAJ_FUSED: one persistent kernel; every trajectory stays in shared memory/registers for its
 *              whole life.  QTRAJ_PLAIN: the plain per-step form, a sequence of separate kernels
 *              over the whole batch per time step with the state in HBM (FP64 only). */
typedef enum { QTRAJ_FUSED = 0, QTRAJ_PLAIN = 1 } qtraj_form;

typedef struct {
    double alpha_s;  /* strong coupling; alpha = C_F alpha_s (Table 1 "alpha"; App. E)            */
    double Nc;       /* number of colours (App. E: C_F = (Nc^2-1)/(2Nc))                         */
    int deriv_type;  /* 0: T = p^2/M; 1: T = 2[1-cos(p dr)]/(M dr^2) (Sec. 2.4, Table 1)          */
    int max_jumps;   /* < 0 unlimited; a jump triggered with n_jumps == max_jumps ends the
                        trajectory with zero overlaps (Sec. 3.5 item 4b)                         */
    double r_max;    /* 1.0 = off; r0 > r_max ends the trajectory with zero overlaps (Sec. 3.5)   */
    int l_cap;       /* < 0 none; a jump to l > l_cap ends the trajectory with zero overlaps
                        (a truncation used to compare with a density matrix cut at l_cap)        */
    int use_rmin;    /* 1: rMin shortcut -- r0 < p_NoJump copies the no-jump result (Sec. 3.5)  */
    int precision;   /* qtraj_precision */
    int form;        /* qtraj_form */
    int save_states; /* 1: keep every final u(r) (FP64) in the workspace for qtraj_states()     */
    int variant;     /* fused kernel variant (FP32, N in {2048, 4096}; elsewhere the same as 0):
                        0 = radix 16, 512 resident threads per SM (384 at N = 4096); 1 = radix 16,
                        640; 2 = radix 8, 768; 3 = radix 8, 1024                                   */
    double t_vacuum; /* >= 0, GeV^-1: vacuum evolution of every initial state before the medium
                        (Table 1: tmed - t0; Sec. 3.5 item 3): round(t_vacuum / dt) Strang steps
                        at T = 0 (Coulomb + centrifugal potential of the state's colour, no
                        imaginary part, no jumps), run once per initial state in qtraj_init, whose
                        result is the state every trajectory starts the medium with and the
                        reference of the survival ratios.  Runs in the fused form of the context's
                        precision, so an FP64 context with t_vacuum > 0 needs N <= 8192. */
    int basis;       /* overlap basis of the observables (App. C; Sec. 2.5): 0 = the analytic Coulomb
                        states u_nl (a0 = 2/(M C_F alpha_s)), discretely normalised; 1 = the numerical
                        eigenstates of the discretised singlet vacuum Hamiltonian of the grid (the
                        propagator's V and kinetic factor), computed at qtraj_create by a
                        preconditioned block eigensolver (the paper's ProjType 1); needs alpha_s > 0. */
    int potential;   /* Table 1 "potential": 0 = the OQS+pNRQCD potential of App. E with quantum jumps;
                        1 = the isotropic KSU potential (App. E, "Isotropic KSU potential"): singlet
                        only, deterministic evolution with H_eff and no jumps (Sec. 2.6: there are no
                        collapse operators for it).  Its real part is the Karsch-Mehr-Satz form with
                        a = 0.409, sigma = 0.21 GeV^2, capped at the vacuum Cornell value at
                        r_SB = 1.25 fm; its imaginary part is -alpha_s C_F T phi(m_D r); m_D =
                        F_mD T sqrt(Nc (1 + N_F/6) pi C_F alpha_s(2 pi T)) with alpha_s(mu) at one
                        loop from alpha_s(5 GeV) = 0.2034 and N_F = 3.  The overlap basis is the
                        numerical eigenstates of the grid's vacuum Hamiltonian with the Cornell
                        potential (basis is ignored), and the survival ratios are the unnormalised
                        |<s|psi>|^2 / |<s|psi_0>|^2 (the norm lost to V_I is the dissociation).
                        Fused form only, no vacuum evolution (t_vacuum = 0), media with Tf >= 0.1 GeV. */
    double ksu_mD_factor; /* F_mD of the KSU Debye mass (> 0; 1 = the perturbative m_D) */
} qtraj_params;

/* Initial state (Table 1, initType/initWidth/initN/initL/initC): kind 0 is the Gaussian
 * u = r^{l+1} exp(-r^2/(2 width^2)); kind 1 is the analytic Coulomb eigenstate (n, l); kind 2 is
 * the numerical eigenstate (n, l) of the discretised singlet vacuum Hamiltonian (initType 100).  color 0 = singlet,
 * 1 = octet.  The state is normalised with the discrete norm (L/N) sum |u_j|^2 = 1 (Eq. normcond). */
typedef struct {
    int kind;
    double width;
    int n, l, color;
} qtraj_init_spec;

/* Medium seen by a trajectory.  kind 0 = Bjorken T(tau) = T0 (tau0/tau)^{1/3} from tau0 until
 * T < Tf (Sec. 3.4, Table 1).  kind 1 = tabulated T(tau) (Table 1 temperatureEvolution 1/2, the
 * file formats of App. B): the points [table_offset, table_offset + table_len) of the context's
 * profile store (qtraj_set_profiles), tau strictly ascending; the medium starts at the first tau,
 * step n uses T linearly interpolated at tau_n = tau_1 + n dt hbar c (the last T past the last
 * point), and it ends after ceil((tau_f - tau_1) / (hbar c dt)) steps, tau_f the first crossing of
 * Tf by the interpolated T (the last tau if T stays >= Tf); T0 and tau0 are ignored.  gamma_hat <= 0
 * and kappa_hat are the transport coefficients
 * kappa = kappa_hat T^3, gamma = gamma_hat T^3 of the potential (App. E).  kappa_hat >= 0 is a
 * constant; kappa_hat = -1, -2, -3 selects the central, lower or upper lattice fit
 * kappa_hat(T) = 1 / (a x^{3/2} + b x + c x^{1/2} + d), x = T / T_c, T_c = 0.155 GeV (App. E, the
 * paper's parameter kappa), evaluated at T(tau_n) every step; a fit requires Tf >= T_c. */
typedef struct {
    int kind;
    double T0, tau0, Tf;
    double kappa_hat, gamma_hat;
    int table_offset, table_len; /* kind 1 only */
} qtraj_medium;

#define QTRAJ_NBASIS 6 /* 1S, 2S, 1P, 3S, 2P, 1D = Coulomb (n,l) (1,0) (2,0) (2,1) (3,0) (3,1) (3,2) */

/* flags of a trajectory record */
#define QTRAJ_F_NOJUMP_SHORTCUT 1 /* r0 < p_NoJump: the no-jump result was copied              */
#define QTRAJ_F_BORDERLINE 2      /* |norm^2 - r| < 1e-12 at some waiting-time comparison      */
#define QTRAJ_F_RMAX 4            /* r0 > r_max                                                */
#define QTRAJ_F_MAXJUMPS 8        /* ended by max_jumps                                        */
#define QTRAJ_F_LCAP 16           /* ended by l_cap                                            */
#define QTRAJ_F_NONFINITE 32      /* norm became NaN/Inf                                       */

/* Result of one trajectory (the ratios.tsv row of App. C plus bookkeeping).  surv[s] is
 * |<s|psi>|^2 / ||psi||^2 divided by |<s|psi_0>|^2, or undivided when the initial overlap is zero
 * (App. C footnote), and 0 unless the final state is a singlet of the basis state's l.
 * jump_digest identifies the whole jump sequence: 32-bit FNV-1a (offset basis 2166136261, prime
 * 16777619) over the bytes, little-endian, of the words (step n, new l, new colour) of every jump in
 * order -- 2166136261 for a trajectory without jumps.  Two runs agree on it exactly when every jump
 * happened at the same step with the same outcome.  192 bytes. */
typedef struct {
    double surv[QTRAJ_NBASIS];
    double ov_re[QTRAJ_NBASIS], ov_im[QTRAJ_NBASIS]; /* <s|psi> of the unnormalised final state */
    double norm2;                                    /* final (L/N) sum |u_j|^2                  */
    double r0;                                       /* the first waiting-time threshold         */
    int l, color, n_jumps, n_steps_exec, flags, first_jump_step;
    int last_jump_step;                              /* step of the last jump, -1 if none        */
    uint32_t jump_digest;                            /* FNV-1a of the jump sequence (above)      */
} qtraj_obs;

/* Create a context for an N-point grid on (0, L] with step dt and heavy-quark mass M (Table 1:
 * num, L, dt, m).  N must be a power of two in [16, 16384] (FP64 fused: <= 8192).  Builds the
 * read-only tables on the current CUDA device (the static potential factors of both colours for
 * l < 256 take 16 KiB x N: 256 MiB at N = 16384); synchronous.  EINVAL on N/L/dt/M/params out of
 * range (alpha_s < 0, Nc < 2, r_max not in (0,1], deriv_type not 0/1, FP32 with the plain form);
 * ENOMEM if the tables do not fit in device memory. */
qtraj_status qtraj_create(int N, double L, double dt, double M, const qtraj_params *params, qtraj_ctx **out);

/* Frees the context and its tables (synchronises the device first).  NULL is a no-op. */
void qtraj_destroy(qtraj_ctx *ctx);

/* Message of the last failing call on this thread ("" if none).  ctx may be NULL. */
const char *qtraj_last_error(const qtraj_ctx *ctx);

/* Device bytes the caller must provide to qtraj_init for n_traj trajectories (records, per-group
 * no-jump results, counters, and the state buffers of the plain form / of save_states). */
size_t qtraj_workspace_bytes(const qtraj_ctx *ctx, int n_traj);

/* Binds the caller's device workspace (>= qtraj_workspace_bytes(ctx, n_traj), 256-byte aligned)
 * and sets the initial states: trajectory t starts in specs[spec_idx[t]] (spec_idx NULL: all use
 * specs[0] when n_specs == 1, else spec t when n_specs == n_traj).  Uploads the normalised initial
 * states and their overlaps with the Coulomb basis (host FP64).  Synchronous.  EINVAL for a spec
 * out of range or an initial state that is not finite or has no positive discrete norm (e.g. a
 * Gaussian whose 2 width^2 underflows to 0). */
qtraj_status qtraj_init(qtraj_ctx *ctx, void *d_workspace, size_t bytes, int n_traj,
                        const qtraj_init_spec *specs, int n_specs, const int *spec_idx);

/* Re-binds the initial state of trajectories [0, n) to specs[spec_idx[t]] of the last qtraj_init,
 * without touching the device (host bookkeeping only; takes effect at the next qtraj_evolve).  Lets a
 * scheduler reuse one bound workspace for batches of different composition.  EINVAL if n exceeds the
 * bound n_traj or an index is out of range. */
qtraj_status qtraj_set_spec_idx(qtraj_ctx *ctx, const int *spec_idx, int n);

/* Copies the context's overlap basis (QTRAJ_NBASIS x N doubles, the order of qtraj_obs.surv) to
 * host memory. */
qtraj_status qtraj_basis_get(const qtraj_ctx *ctx, double *out);

/* One row of the per-step summary of a trajectory (App. C, summary.tsv): after step `step` (1-based
 * count of the medium's steps), before a jump triggered at that step -- the discrete norm^2, the
 * colour and l, the overlaps |<nl|psi>|^2 / norm^2 with the Coulomb basis (zero unless a singlet of
 * the basis state's l) and R = <psi|r|psi> / norm^2 / <1S|r|1S>.  80 bytes. */
typedef struct {
    int step, color, l, flags;
    double norm2;
    double ov2[6];
    double r_ratio;
} qtraj_trace_rec;

/* Turns the per-step summary on (every > 0) or off (every = 0) for the evolves that follow: the first
 * n_traced trajectories of each batch write a row every `every` steps and after their last step, at
 * most max_records rows each, to d_records[t * max_records + i]; d_counts[t] receives the number of
 * rows (the evolve clears d_counts[0 .. n_traced) first).  Both are caller device buffers that must
 * stay valid while those evolves run.  A trajectory resolved without evolving (rMin shortcut,
 * r_max) writes no row.  Fused form only (EINVAL for the plain form); while it is on, evolves run a
 * traced copy of the fused kernel (variant 0's plan), which at each recorded step of a traced
 * trajectory makes one more pass over the state per quantity. */
qtraj_status qtraj_set_trace(qtraj_ctx *ctx, int every, int n_traced, int max_records, qtraj_trace_rec *d_records,
                             int *d_counts);

/* Sets the context's profile store: n_points (tau [fm/c], T [GeV]) points from host arrays,
 * referred to by kind-1 media through (table_offset, table_len).  Several profiles share the store
 * back to back.  Waits for the context's queued work, then uploads (synchronous); replaces the
 * previous store.  EINVAL for n_points < 2 or a non-finite or negative value. */
qtraj_status qtraj_set_profiles(qtraj_ctx *ctx, const double *tau, const double *T, int n_points);

/* Evolves trajectories [0, batch) of the bound workspace through their media: trajectory t sees
 * media[medium_idx[t]] (same NULL rule as qtraj_init) and draws its waiting-time thresholds and
 * jump choices from Philox4x32-10 keyed by seeds[t] (host array of batch entries).  With use_rmin,
 * also evolves one no-jump trajectory per distinct (initial state, medium) pair (the rMin shortcut,
 * Sec. 3.5 item 4a): the plain form runs them first; the fused form runs them as the first work
 * items of its single launch, and a trajectory taken up after its group's no-jump record is
 * published, with r0 < p_NoJump, copies it (QTRAJ_F_NOJUMP_SHORTCUT, n_steps_exec = 0), while one
 * taken up before evolves its whole medium -- the same record, since the shortcut is exact, with its
 * steps counted.  Asynchronous on `stream`; results are read with qtraj_observables. */
qtraj_status qtraj_evolve(qtraj_ctx *ctx, int batch, const qtraj_medium *media, int n_media, const int *medium_idx,
                          const uint64_t *seeds, void *stream);

/* Copies the batch's qtraj_obs records (batch x sizeof(qtraj_obs) bytes) to `out` (host memory if
 * out_is_device == 0, then the call synchronises `stream`; device memory otherwise).  Returns
 * QTRAJ_ENONFINITE after a host copy if any trajectory's norm became non-finite. */
qtraj_status qtraj_observables(qtraj_ctx *ctx, void *out, int out_is_device, void *stream);

/* Copies the final states (batch x N complex128, u_0 = 0) saved with params.save_states = 1. */
qtraj_status qtraj_states(qtraj_ctx *ctx, void *out, int out_is_device, void *stream);

/* The no-jump results (p_NoJump = norm2) of the last evolve, one per (init spec, medium) pair in
 * spec-major order (n_specs x n_media records; pairs not used are zero).  Synchronises. */
qtraj_status qtraj_nojump_results(qtraj_ctx *ctx, qtraj_obs *out_host, int capacity, int *n_written);

/* Counters of the last evolve: steps executed (sum over trajectories, including the no-jump runs),
 * trajectories run / short-cut, kernel launches, and the device time of the step kernels measured
 * with events on the caller's stream (valid after a synchronising call): ms_nojump is the plain
 * form's separate no-jump phase (0 for the fused form, whose no-jump runs share the main launch). */
typedef struct {
    int64_t steps_executed;
    int64_t nojump_steps;
    int n_traj, n_shortcut, n_groups;
    int launches;
    float ms_nojump, ms_main;
} qtraj_run_stats;
qtraj_status qtraj_last_run_stats(qtraj_ctx *ctx, qtraj_run_stats *out);

/* Launch geometry of the fused kernel for this context (threads per trajectory, CTAs per SM,
 * dynamic shared memory per CTA, registers per thread). */
typedef struct {
    int threads_per_traj, ctas_per_sm, smem_bytes, regs_per_thread, radix, sm_count;
} qtraj_kernel_info;
qtraj_status qtraj_kernel_info_get(const qtraj_ctx *ctx, qtraj_kernel_info *out);

/* Measurement of the radix-16 DFT blocks of the sine transforms (Sec. 3.3; the paper's transforms
 * are FFTW calls and have no tensor-core form): one CTA per batch of 256 columns of 16 complex FP32
 * points, resident in shared memory, applies `passes` times y = (F/4) x to every column, F the
 * 16-point DFT matrix exp(-2 pi i m'm/16) ((F/4)^4 = I).  method 0: CUDA cores (the fused kernel's
 * DFT16, constants in hi+lo, then times 1/4).  Tensor cores, mma.sync -> FP32 with the matrix in PA
 * parts, each value in PB parts and the products of part orders j + k <= MAXORD: 1 BF16X3 (BF16,
 * PA = PB = 2, 3 products); 2 BF16X9 (BF16, PA = 4, PB = 3, 9 products); 3 FP16X3 (FP16, PA = PB = 2,
 * 3 products); 4 FP16X5 (FP16, PA = 3, PB = 2, 5 products); the FP16 forms scale each column by a
 * power of two before the split.  x_host: n_batches x 256 x 16 complex values as (re, im) doubles,
 * point m of column c of batch b at ((b 256 + c) 16 + m), converted to FP32; y_host (same layout)
 * receives the result; *ms the device time of the timed launch, which follows one untimed launch.
 * Synchronous; allocates and frees its device buffers.  QTRAJ_EINVAL for a method outside 0..4,
 * n_batches <= 0, passes < 0 or a null buffer; QTRAJ_ECUDA with the CUDA error's text. */
qtraj_status qtraj_dft16_study(int method, int n_batches, int passes, const double *x_host, double *y_host,
                               double *ms);

/* ---------------------------------------------------------------------------------------------
 * Serving: continuous batching of trajectory requests.  (The paper has no counterpart: its program
 * evolves one batch per invocation.)
 *
 * A server owns, for every grid size N it serves, `slots_per_n` contexts, each with its share of
 * the caller's workspace, its own non-blocking CUDA stream and a pinned host buffer for results.
 *   - qtraj_submit queues a request: n trajectory descriptors (grid size, initial state from the
 *     server's catalogue, medium, Philox seed) under a caller-chosen id.  Host only.
 *   - qtraj_poll never blocks.  It collects finished launches; admits queued requests first come
 *     first served while the trajectories admitted and not yet returned stay within
 *     max_inflight_traj (a request larger than the whole budget is admitted when nothing else is in
 *     flight); and fills every idle slot with up to waves_per_launch waves (SMs x resident CTAs)
 *     of trajectories taken across the admitted requests of that grid size in the order `order`
 *     sets (arrival, or least work first).  So the
 *     trajectories of several requests share a launch, a request that arrives while others run
 *     joins the next launch that frees up, and slots of different grid sizes run concurrently on the
 *     device.  It writes to done_ids the ids of requests whose last trajectory has finished (at
 *     most `capacity`; the rest are reported by the next call).
 *   - qtraj_request_result copies a finished request's n records (in submission order) to host
 *     memory and forgets the request.
 * A trajectory's record depends only on its descriptor, never on its launch mates.  Every launch
 * is the fused form with the rMin shortcut off (launches mix many (state, medium) groups); the
 * other fields of `params` apply.  Media are Bjorken (kind 0; a lattice-fit kappa_hat is allowed);
 * tabulated profiles need a context's profile store and are not served.  Errors: QTRAJ_EINVAL for
 * a grid size not served, a catalogue index out of range, an invalid medium (as in qtraj_evolve;
 * kind 1 always, the slots having no profile store), n <= 0, or an id already queued or
 * not yet returned (checked in qtraj_submit, before anything is queued); QTRAJ_ECUDA from qtraj_poll
 * if a launch failed, after which the requests of that launch never finish and the server is to be
 * destroyed.  One host thread at a time per server.
 * --------------------------------------------------------------------------------------------- */
typedef struct qtraj_server qtraj_server;

typedef struct {
    int N;               /* grid size: one of the server's */
    int spec;            /* index into the server's initial-state catalogue */
    qtraj_medium medium; /* this trajectory's medium */
    uint64_t seed;       /* Philox key (Sec. 3.5 draws) */
} qtraj_traj_desc;

typedef struct {
    const int *Ns;                 /* grid sizes served (powers of two, 16..16384); L = N * dr */
    int n_N;
    double dr, dt, M;              /* grid spacing (GeV^-1), step (GeV^-1), heavy-quark mass (GeV) */
    const qtraj_params *params;    /* physics options and precision; form, save_states, use_rmin ignored */
    const qtraj_init_spec *specs;  /* initial-state catalogue, 1..QTRAJ_SERVER_MAX_SPECS entries */
    int n_specs;
    int slots_per_n;               /* contexts per grid size, >= 1 */
    int waves_per_launch;          /* >= 1 */
    int64_t max_inflight_traj;     /* admission budget, >= 1 */
    int order;                     /* which admitted trajectories of a grid size fill a launch first:
                                      QTRAJ_ORDER_ARRIVAL (0, requests in arrival order) or
                                      QTRAJ_ORDER_SHORTEST (1, requests of least work first, the work
                                      of a request being sum N log2 N x steps of its trajectories;
                                      ties in arrival order) */
} qtraj_server_config;
#define QTRAJ_ORDER_ARRIVAL 0
#define QTRAJ_ORDER_SHORTEST 1

/* One launch of a server slot: its grid size, trajectories and requests, and its device start and end
 * (events on the slot's stream around the evolve) in ms since qtraj_server_create. */
typedef struct {
    int N, n_traj, n_requests, pad;
    double start_ms, end_ms;
} qtraj_launch_rec;

#define QTRAJ_SERVER_MAX_SPECS 64

/* Device workspace the server needs (bytes, 256-byte aligned base required). */
qtraj_status qtraj_server_workspace_bytes(const qtraj_server_config *cfg, size_t *bytes);
/* Creates the contexts, binds them to d_ws and uploads the catalogue's initial states.  Synchronous. */
qtraj_status qtraj_server_create(const qtraj_server_config *cfg, void *d_ws, size_t bytes, qtraj_server **out);
qtraj_status qtraj_submit(qtraj_server *srv, const qtraj_traj_desc *traj, int n, uint64_t request_id);
qtraj_status qtraj_poll(qtraj_server *srv, uint64_t *done_ids, int capacity, int *n_done);
qtraj_status qtraj_request_result(qtraj_server *srv, uint64_t request_id, qtraj_obs *out, int n);
/* Requests queued but not admitted, admitted but not finished, and launches in flight. */
qtraj_status qtraj_server_counts(const qtraj_server *srv, int *waiting, int *admitted, int *launches_in_flight);
/* The finished launches recorded since the server was created (or since the last call with
 * clear = 1), oldest first: up to `capacity` records into out (host), *n_written set.  Host only;
 * a launch is recorded when qtraj_poll retires it. */
qtraj_status qtraj_server_launch_log(qtraj_server *srv, qtraj_launch_rec *out, int capacity, int *n_written, int clear);
/* Waits for the launches in flight, then frees everything the server allocated (not d_ws). */
void qtraj_server_destroy(qtraj_server *srv);

/* ---------------------------------------------------------------------------------------------
 * Evolving without allocating.  (The paper has no counterpart: its program runs on CPUs only.)
 *
 * For callers that cannot allocate at the point of the call -- a service that hands all device
 * memory to its own pool at start-up and must not touch the CUDA allocator afterwards, or a
 * latency-bound loop in which an allocation could synchronise the device or fail under
 * fragmentation.  qtraj_evolve_static runs the fused form (the context's precision and options)
 * for `batch` trajectories given entirely by host arrays -- initial-state specs with a per-trajectory
 * index, media with a per-trajectory index (NULL index: as in qtraj_init/qtraj_evolve), seeds -- and
 * writes batch qtraj_obs records to the device buffer d_out.  It needs no qtraj_init and no
 * workspace, and it calls no cudaMalloc, cudaFree, cudaMallocHost or any other allocating routine:
 * every intermediate lives in one fixed device array inside the library (about 2 MB, held by every
 * device that loads the library until the process exits) and in fixed host arrays.
 *
 * Limits: batch <= QTRAJ_STATIC_MAX_TRAJ, n_specs <= QTRAJ_STATIC_MAX_SPECS,
 * n_media <= QTRAJ_STATIC_MAX_MEDIA, N <= 16384; larger requests return QTRAJ_EINVAL with a message.
 * The first call on a device looks up the device address of that array (cudaGetSymbolAddress) with
 * the device current; make that first call before any stream capture.  All calls share the one array
 * (the work counter and status word are cleared by every call): calls whose GPU work overlaps -- on
 * different streams, or from different host threads without ordering -- race on it and must be
 * serialised by the caller (the host side of the call is serialised by a lock).  The context's
 * device must be the current device (QTRAJ_EINVAL otherwise).  The call copies its inputs to the
 * device array from the library's fixed host arrays, which are pageable memory: each copy first
 * waits for the work already queued on `stream`, so the call returns once earlier work on `stream`
 * has finished and its inputs are on their way; the evolve itself is then queued on `stream` and
 * not waited for.  The caller's host arrays may be reused when the call returns.  An initial state
 * that is not finite or has no positive norm (e.g. a Gaussian whose 2 width^2 underflows) is
 * refused with QTRAJ_EINVAL before any GPU work.
 * --------------------------------------------------------------------------------------------- */
#define QTRAJ_STATIC_MAX_TRAJ 4096
#define QTRAJ_STATIC_MAX_SPECS 8
#define QTRAJ_STATIC_MAX_MEDIA 64
qtraj_status qtraj_evolve_static(qtraj_ctx *ctx, int batch, const qtraj_init_spec *specs, int n_specs,
                                 const int *spec_idx, const qtraj_medium *media, int n_media, const int *medium_idx,
                                 const uint64_t *seeds, qtraj_obs *d_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* QTRAJ_H */
