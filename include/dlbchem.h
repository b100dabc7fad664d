/*
 * dlbchem: batched stiff chemistry for the operator-split reacting-flow step,
 * GB300 (sm_103a) CUDA library with a plain C ABI.
 *
 * The problem (DLBFoam paper, arXiv 2011.07978, Sec. 1 and Sec. 2.1): after
 * operator splitting, every CFD cell n carries an independent stiff ODE
 * dPhi/dt = f(Phi) for its thermochemical state Phi = (T, p, Y) over one flow
 * step dt, and the cost of each cell depends on its initial state. Here p is
 * held constant and the mixture is an adiabatic ideal gas, so each cell
 * integrates y = (T, Y_1..Y_nsp) with mass-action Arrhenius kinetics, reverse
 * rates from equilibrium constants built on species Gibbs energies, and
 * third-body reactions. The integrator is the L-stable 4-stage Rosenbrock
 * method of Hairer and Wanner (Solving ODEs II, Sec. IV.7) with embedded
 * error estimate and adaptive steps, run by one warp (or one 4-warp team)
 * per cell.
 *
 * The paper's two speed-ups become on-device scheduling here:
 *  - load balancing (Sec. 2.2, Algorithm 1): cells are ordered by a cost key
 *    (the per-cell step count of the previous call, the analogue of the
 *    per-cell CPU time t_cpu^n) and pulled by a persistent kernel from a
 *    device work queue, longest first;
 *  - reference mapping (Sec. 2.3): cells close to a reference state reuse
 *    the solution of the first such cell instead of being integrated.
 *
 * Conventions for every entry point:
 *  - Arrays are species-major structure-of-arrays: Y[k * ncells + i] is the
 *    mass fraction of species k in cell i. T in K, p in Pa.
 *  - Unless a function says otherwise, pointers are DEVICE pointers owned by
 *    the caller, and the work is enqueued asynchronously on the CUDA stream
 *    passed as `cuda_stream` (a cudaStream_t; NULL = legacy default stream).
 *  - Return codes cover argument validation and launch errors only; per-cell
 *    outcomes are in status[] (device memory) once the stream has reached
 *    the end of the call.
 *  - A context is not thread-safe: calls on one context must not overlap on
 *    the host. Calls on different contexts are independent.
 */
#ifndef DLBCHEM_H
#define DLBCHEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define DLBCHEM_OK 0
#define DLBCHEM_BAD_ARG 1   /* an argument is out of range or a pointer is NULL */
#define DLBCHEM_BAD_MECH 2  /* mechanism file missing, truncated or inconsistent */
#define DLBCHEM_CUDA 3      /* a CUDA runtime call or kernel launch failed */
#define DLBCHEM_OOM 4       /* device workspace allocation failed */

/* Per-cell status[] values. */
#define DLBCHEM_CELL_OK 0
#define DLBCHEM_CELL_MAPPED 1          /* copied the reference cell's increment */
#define DLBCHEM_CELL_SURROGATE 2       /* the network's increment passed the gate */
#define DLBCHEM_CELL_MAX_STEPS (-1)    /* max_steps attempted steps reached */
#define DLBCHEM_CELL_H_UNDERFLOW (-2)  /* step size fell below hmin_frac*dt */
#define DLBCHEM_CELL_NONFINITE (-3)    /* input not finite, T <= 0 or p <= 0 */
/* A failed cell returns its last accepted state in T_out / Y_out. */

/* Scheduling modes (dlbchem_options.schedule). */
#define DLBCHEM_SCHED_PLAIN 0   /* one team per cell, cells in index order */
#define DLBCHEM_SCHED_QUEUE 1   /* persistent teams pull cells longest-first */

typedef struct dlbchem_ctx dlbchem_ctx;

/*
 * Integration and scheduling options. Sec. 4.1 of the paper gives the ODE
 * tolerances rtol/atol; Sec. 2.3 the mapping tolerances (read here as a
 * composition tolerance on max_k |Y_k - Yref_k| and a relative temperature
 * tolerance |T - T_ref| < map_Ttol * T_ref).
 */
typedef struct dlbchem_options {
  double rtol;          /* relative tolerance of the error norm (default 1e-6) */
  double atol;          /* absolute tolerance (default 1e-10) */
  int32_t max_steps;    /* attempted steps per cell before MAX_STEPS (100000) */
  int32_t isothermal;   /* 1: freeze T (f_T = 0) */
  double hmin_frac;     /* H_UNDERFLOW when h < hmin_frac * dt (1e-20) */
  int32_t schedule;     /* DLBCHEM_SCHED_PLAIN or DLBCHEM_SCHED_QUEUE */
  int32_t chunk;        /* cells per queue pull (1) */
  int32_t mapping;      /* 0: off; 1: one reference cell (the lowest-index cell within
                           tolerance of Yref, Sec. 2.3); 2: one reference per state bucket
                           (Sec. 2.3 generalised): the bucket key is (the IEEE bits of T
                           shifted right by s, s the largest with 2^(s-52) <= map_Ttol;
                           floor(Y_k / map_Ytol) per species), the reference is the bucket's
                           lowest-index eligible cell (finite state, T > 0, T < map_Tmax if
                           set), and a cell maps when the keys agree and it meets the Sec. 2.3
                           criterion against it. Mapped cells get T' = T'_r + (T - T_r),
                           Y' = Y'_r + (Y - Y_r): the reference's increment. */
  int32_t timing;       /* 1: record CUDA events around each kernel (see dlbchem_last_timing) */
  double map_Ttol;      /* relative temperature tolerance (1e-4) */
  double map_Ytol;      /* absolute composition tolerance (1e-4) */
  double map_Tmax;      /* > 0: only cells below this T qualify (0 = off) */
  int32_t team_warps;   /* warps per cell: 1, 2, 4, or 0 = automatic (1 up to 32 unknowns, 2 up to 64, else 4) */
  int32_t precision;    /* 0: FP64 LU of the iteration matrix (default); 1: FP32 LU with FP64
                           iterative refinement: residuals against the FP64 matrix, stopped when
                           the estimated remaining error is below 1e-6 of the error weights, at
                           most 3 rounds, the step redone with the FP64 LU if they do not
                           converge. State, rates, error norm and step control stay FP64.
                           Fixed at create, which then allocates one FP64 matrix copy per
                           resident team (SMs x CTAs per SM x teams x N^2 doubles; 22 MB at 54
                           unknowns on 152 SMs); integrations of such a context always launch
                           persistent teams (the plain schedule keeps index order). */
  int32_t predictor;    /* 1: order the queue by the attached network's predicted step counts
                           (no previous call needed); steps[] is then only written */
  int32_t surrogate;    /* 1: try the attached network's increments first; cells that pass the
                           gate get status DLBCHEM_CELL_SURROGATE, the others are integrated;
                           2: candidates y + dt f(y) + the network's output (an explicit Euler
                           step corrected by a network trained on the residual increment
                           - dt f(y), see dlbchem_rhs), then y + dt f(y), then y */
  double gate;          /* surrogate gate tolerance (default 1e-4): trapezoid defect per mass
                           fraction (relative for T), |sum Y' - 1|, relative element change,
                           every Y'_k >= -gate, and dt |f(y') - f(y)| <= |y' - y| + 2 gate
                           (not stiff along the increment) */
} dlbchem_options;

/* Fill *opt with the defaults listed above. Returns DLBCHEM_OK or BAD_ARG. */
int dlbchem_options_default(dlbchem_options* opt);

/*
 * Load a mechanism file (the DLBMECH1 binary format written by the seeded
 * generator: species thermo, Arrhenius reactions with third bodies and
 * listed efficiencies, and optional fall-off (Lindemann, Troe), PLOG and
 * NASA-7 thermo sections; synth/mechfile.py documents the layout) on the
 * current CUDA device and create a context: the
 * preprocessing of Sec. 2.2 stage 1 that every cell shares (the kinetics
 * each problem of Sec. 2.2 is integrated with). opt may be
 * NULL (defaults). On success *out owns device copies of the mechanism
 * tables; release it with dlbchem_destroy. On failure *out is NULL and the
 * message is available from dlbchem_last_error(NULL).
 * Returns DLBCHEM_OK, BAD_ARG, BAD_MECH, CUDA or OOM.
 */
int dlbchem_create(const char* mech_path, const dlbchem_options* opt, dlbchem_ctx** out);

/* Replace the context's options (validated; BAD_ARG leaves them unchanged). */
int dlbchem_set_options(dlbchem_ctx* ctx, const dlbchem_options* opt);

/*
 * Integrate ncells independent cells over one flow step dt (paper Sec. 2.2,
 * stage 3, with stages 1 and 4 fused around it).
 *   T, p   [ncells] inputs; Y [nsp][ncells] input mass fractions.
 *   T_out  [ncells], Y_out [nsp][ncells] results; may alias T / Y.
 *   steps  [ncells] int32, nullable. If non-NULL it is read first as the
 *          per-cell cost key of the queue (the previous call's counts, the
 *          analogue of t_cpu^n in Algorithm 1; all-zero keys give index
 *          order) and then overwritten with the attempted steps of this call
 *          (accepted + rejected; 0 for mapped cells).
 *   status [ncells] int32, nullable: per-cell DLBCHEM_CELL_* codes.
 *   Yref   [nsp] device pointer, nullable: the reference composition of the
 *          mapping criterion with mapping 1; NULL uses cell 0's composition.
 *          Ignored with mapping 2.
 * ncells == 0 is a no-op. Mapping and the queue follow ctx's options.
 * Returns DLBCHEM_OK, BAD_ARG (NULL pointer, dt <= 0 or not finite, ncells
 * < 0), CUDA or OOM (workspace growth failed).
 */
int dlbchem_integrate(dlbchem_ctx* ctx, int64_t ncells, double dt, const double* T, const double* p,
                      const double* Y, double* T_out, double* Y_out, int32_t* steps, int32_t* status,
                      const double* Yref, void* cuda_stream);

/*
 * Same as dlbchem_integrate, but every array is a HOST pointer (pageable or
 * pinned). The call copies the inputs into a device staging area owned by
 * the context, integrates, copies the results back and synchronises the
 * stream before returning. steps may be NULL (no cost key); status may be
 * NULL. Returns as dlbchem_integrate.
 */
int dlbchem_integrate_host(dlbchem_ctx* ctx, int64_t ncells, double dt, const double* T, const double* p,
                           const double* Y, double* T_out, double* Y_out, int32_t* steps, int32_t* status,
                           const double* Yref, void* cuda_stream);

/*
 * Queued integration that allocates nothing (the paper has no counterpart:
 * this serves callers, not the method). For flow solvers that reserve all
 * device memory up front (their own pool, a fixed budget per GPU) and may not
 * call cudaMalloc in their time loop, where it can fail once the pool owns
 * the device and where it synchronises the whole device: dlbchem_integrate
 * grows its scratch with cudaMalloc when a larger field arrives, this call
 * never does.
 * Same arguments and results as dlbchem_integrate with the queue schedule,
 * cost keys from steps (sorted longest first when steps is non-NULL) and no
 * mapping, whatever ctx's options say about schedule and mapping; the other
 * options (tolerances, max_steps, isothermal, chunk, precision) apply.
 * Its scratch is one array of 5.3 MB compiled into the library, for up to
 * DLBCHEM_STATIC_MAX_CELLS cells; larger ncells returns BAD_ARG. CUDA loads
 * that array lazily; dlbchem_create loads it on ctx's device, which holds it
 * from then until the process exits (if that load failed, the first static
 * call on the device loads it and reports a failure as CUDA). ctx's device
 * must be current. All calls share the array and each call clears what it
 * needs, so calls that overlap on the GPU race and must be serialised by the
 * caller. After the call, dlbchem_last_stats describes it (no mapped cells)
 * and dlbchem_last_worklist / dlbchem_last_timing report nothing.
 * Returns DLBCHEM_OK, BAD_ARG or CUDA.
 */
#define DLBCHEM_STATIC_MAX_CELLS 262144
int dlbchem_integrate_static(dlbchem_ctx* ctx, int64_t ncells, double dt, const double* T, const double* p,
                             const double* Y, double* T_out, double* Y_out, int32_t* steps, int32_t* status,
                             void* cuda_stream);

/*
 * Batched uneven launch (several meshes of uneven sizes over several
 * mechanisms; the paper's balancing across processes, Sec. 2.2, becomes one
 * device queue per mechanism). Meshes that share a mechanism file form a
 * class; each class runs as ONE persistent integrator launch whose work list
 * spans all its meshes, longest first by the previous call's steps[]; the
 * classes run on forked streams inside ONE captured CUDA graph.
 *   dlbchem_batch_create  options common to all meshes (tolerances, ...);
 *   dlbchem_batch_add     registers a mesh: mechanism path, ncells (< 2^27),
 *                         its own dt and DEVICE arrays as in
 *                         dlbchem_integrate (steps nullable: cost keys in,
 *                         counts out; status nullable). At most 8 meshes per
 *                         mechanism and 8 mechanisms. The arrays must stay
 *                         valid while the graph exists (they are baked in).
 *   dlbchem_batch_tune    autotuner: for each class, times every (team
 *                         warps in {1,2,4}, queue chunk in {1,4,16}) on a
 *                         sample of about sample_cells cells (prefixes of its
 *                         meshes, whose outputs it overwrites) and keeps the
 *                         fastest; results are cached per (species,
 *                         reactions, dt) for the process. Synchronous.
 *   dlbchem_batch_capture allocates the engines and workspaces, then
 *                         captures the graph on `cuda_stream` (non-NULL).
 *   dlbchem_batch_launch  replays the graph on `cuda_stream`.
 *   dlbchem_batch_info    class i: out[0] meshes, out[1] cells, out[2] team
 *                         warps, out[3] queue chunk, out[4] species,
 *                         out[5] tuned sample time in microseconds (-1: untuned).
 * Return DLBCHEM_OK, BAD_ARG, BAD_MECH, CUDA or OOM; the message is in
 * dlbchem_batch_last_error.
 */
typedef struct dlbchem_batch dlbchem_batch;
int dlbchem_batch_create(const dlbchem_options* opt, dlbchem_batch** out);
int dlbchem_batch_add(dlbchem_batch* b, const char* mech_path, int64_t ncells, double dt, const double* T,
                      const double* p, const double* Y, double* T_out, double* Y_out, int32_t* steps,
                      int32_t* status);
int dlbchem_batch_tune(dlbchem_batch* b, int64_t sample_cells, void* cuda_stream);
int dlbchem_batch_capture(dlbchem_batch* b, void* cuda_stream);
int dlbchem_batch_launch(dlbchem_batch* b, void* cuda_stream);
int dlbchem_batch_info(dlbchem_batch* b, int cls, int64_t out[6]);
const char* dlbchem_batch_last_error(const dlbchem_batch* b);
void dlbchem_batch_destroy(dlbchem_batch* b);

/*
 * Learned cost predictor and surrogate (the paper has no counterpart; it
 * replaces the per-cell CPU time of the last step, Algorithm 1's t_cpu^n, by
 * a prediction, and adds an error-gated shortcut). A multilayer perceptron
 * n_in -> n_hidden -> n_hidden -> n_hidden -> n_out with SiLU, trained and run
 * by the library's BF16 tensor-core kernels with FP32 accumulation. For a
 * mechanism with nsp species: n_in = nsp + 3 (T/1000, ln p, Y, ln dt), n_out =
 * nsp + 2 (ln attempted steps, dT, dY), each normalised by the stored means
 * and standard deviations.
 *   create / destroy / nparams; set_params / get_params copy the flat FP32
 *   parameter vector [W1 b1 W2 b2 W3 b3 W4 b4] (W row-major [fan_in][fan_out])
 *   from / to DEVICE memory and reset the optimiser; set_norm takes HOST
 *   arrays mu_x, sd_x [n_in] and mu_y, sd_y [n_out].
 *   forward: X [batch][n_in] -> out [batch][n_out], normalised, device. Where
 *   the hidden width is a multiple of 64 up to 256 and n_in, n_out <= 256 it
 *   runs the whole network in one kernel per 128 rows (activations stay in
 *   shared memory, weights stream in as packed BF16 tiles), else layer by
 *   layer; both give the same BF16/FP32 arithmetic. set_fused(m, 0) forces
 *   the layer-by-layer forward, set_fused(m, 1) restores the default
 *   (BAD_ARG otherwise); fused(m) is 1 when forward takes the whole-network
 *   kernel, 0 when not, -1 for NULL.
 *   grad: MSE loss and its gradient (grad device [nparams] or NULL for the
 *   internal buffer; loss device float or NULL). adam: one Adam step
 *   (Kingma & Ba 2015) with the given or the internal gradient.
 *   train_step = grad + adam on the internal gradient.
 *   dlbchem_attach_mlp: the network ctx uses when options.predictor or
 *   options.surrogate is on (NULL detaches). The network must outlive its use.
 * Return DLBCHEM_OK, BAD_ARG, CUDA or OOM (message: dlbchem_mlp_last_error).
 */
typedef struct dlbchem_mlp dlbchem_mlp;
int dlbchem_mlp_create(int n_in, int n_hidden, int n_out, dlbchem_mlp** out);
int64_t dlbchem_mlp_nparams(const dlbchem_mlp* m);
int dlbchem_mlp_set_params(dlbchem_mlp* m, const float* params, void* cuda_stream);
int dlbchem_mlp_get_params(dlbchem_mlp* m, float* params, void* cuda_stream);
int dlbchem_mlp_set_norm(dlbchem_mlp* m, const float* mu_x, const float* sd_x, const float* mu_y, const float* sd_y);
int dlbchem_mlp_forward(dlbchem_mlp* m, int64_t batch, const float* X, float* out, void* cuda_stream);
int dlbchem_mlp_grad(dlbchem_mlp* m, int64_t batch, const float* X, const float* Y, float* grad, float* loss,
                     void* cuda_stream);
int dlbchem_mlp_adam(dlbchem_mlp* m, const float* grad, float lr, void* cuda_stream);
int dlbchem_mlp_train_step(dlbchem_mlp* m, int64_t batch, const float* X, const float* Y, float lr, float* loss,
                           void* cuda_stream);
int dlbchem_mlp_set_fused(dlbchem_mlp* m, int enable);
int dlbchem_mlp_fused(const dlbchem_mlp* m);
const char* dlbchem_mlp_last_error(const dlbchem_mlp* m);
void dlbchem_mlp_destroy(dlbchem_mlp* m);
int dlbchem_attach_mlp(dlbchem_ctx* ctx, dlbchem_mlp* m);

/* Number of species / reactions of the loaded mechanism (-1 if ctx NULL): the
 * size of the per-cell state (Sec. 2.2: a problem carries N_sp + 6 doubles)
 * and of the kinetics. */
int dlbchem_nspecies(const dlbchem_ctx* ctx);
int dlbchem_nreactions(const dlbchem_ctx* ctx);

/*
 * Statistics of the last completed call on ctx (synchronises its stream).
 *   out[0] cells integrated, out[1] cells mapped (or taken from the
 *   surrogate), out[2] reference cell index with mapping 1 (-1 if none or
 *   with mapping 2; see dlbchem_last_mapping), out[3] team size in threads, out[4] teams per CTA,
 *   out[5] CTAs launched by the integrator, out[6] dynamic shared memory
 *   bytes per CTA, out[7] kernel launches in the call, out[8] steps whose
 *   FP32 refinement fell back to the FP64 LU, out[9] precision mode.
 * Returns DLBCHEM_OK, BAD_ARG or CUDA.
 */
int dlbchem_last_stats(dlbchem_ctx* ctx, int64_t out[10]);

/*
 * Device time of the kernels of the last call, in milliseconds, measured with
 * CUDA events recorded on the call's stream around each launch when the
 * context was created (or set) with options.timing = 1; 0 otherwise.
 *   out[0] integrator (Rosenbrock) kernel, out[1] mapping classification,
 *   out[2] cost-key sort, out[3] mapping scatter, out[4..7] reserved.
 * Synchronises the stream of the last call. Returns DLBCHEM_OK or BAD_ARG.
 */
int dlbchem_last_timing(dlbchem_ctx* ctx, double out[8]);

/*
 * Diagnostic: copy the work list of the last call (the cells handed to the
 * integrator, in the order the queue hands them out: unmapped cells sorted
 * by descending cost key, ties in index order) into list_out, a DEVICE
 * array of at least ncells int32, and its length into *m_out (host).
 * Only valid after a call with mapping or the queue schedule; otherwise
 * *m_out = -1. Synchronises the stream of the last call.
 * Returns DLBCHEM_OK, BAD_ARG or CUDA.
 */
int dlbchem_last_worklist(dlbchem_ctx* ctx, int32_t* list_out, int64_t* m_out);

/*
 * Which cells the last call mapped, and to which reference (Sec. 2.3): writes
 * ref_out[i] = the reference cell of mapped cell i, -1 for every other cell,
 * into ref_out, a DEVICE array of at least ncells int32, and ncells into
 * *n_out (host). Only valid after a call with mapping 1 or 2; otherwise
 * *n_out = -1. Runs on and synchronises the stream of the last call.
 * Returns DLBCHEM_OK, BAD_ARG or CUDA.
 */
int dlbchem_last_mapping(dlbchem_ctx* ctx, int32_t* ref_out, int64_t* n_out);

/*
 * Diagnostic: evaluate the integrator's own exponential (Tang's table-driven
 * method) and reciprocal (one third-order correction of the hardware estimate)
 * next to CUDA's exp and IEEE division. x [n] device input; out [4n] device
 * output, per element: exp_own, exp_cuda, rcp_own, 1/x. Asynchronous on the
 * stream. Returns DLBCHEM_OK, BAD_ARG or CUDA.
 */
int dlbchem_check_math(dlbchem_ctx* ctx, int64_t n, const double* x, double* out, void* cuda_stream);

/*
 * Right-hand side of every cell's ODE (Sec. 1: the thermochemical state
 * evolves by dPhi/dt = f(Phi); here f = (dT/dt, dY_k/dt) of a constant-
 * pressure ideal gas with the mechanism's rates, isothermal per ctx's
 * options). T, p [ncells], Y [nsp][ncells] device inputs; fT [ncells],
 * fY [nsp][ncells] device outputs (K/s, 1/s). Cells with a non-finite state,
 * T <= 0 or p <= 0 get NaN. Asynchronous on the stream.
 * Returns DLBCHEM_OK, BAD_ARG or CUDA.
 */
int dlbchem_rhs(dlbchem_ctx* ctx, int64_t ncells, const double* T, const double* p, const double* Y, double* fT,
                double* fY, void* cuda_stream);

/*
 * Measurement aid (not a step of the method): FP64 FMA throughput probe, the
 * measured denominator of the integrator's FP64 roofline fraction. Launches
 * nout / 256 blocks of 256 threads; every thread runs `iters` rounds of eight
 * independent FP64 FMA chains and writes one value to out[nout] (device,
 * nout a positive multiple of 256). *flops receives the launch's FP64 flop
 * count (2 per FMA); time the launch with events on the same stream.
 * Asynchronous. Returns DLBCHEM_OK, BAD_ARG or CUDA.
 */
int dlbchem_fp64_fma_probe(int64_t iters, double* out, int64_t nout, int64_t* flops, void* cuda_stream);

/* Message of the last failed call on ctx, or of the last failed create when
 * ctx is NULL. Never NULL; "" when there was no error. Owned by the library.
 * (Bookkeeping of the library; the paper has no counterpart.) */
const char* dlbchem_last_error(const dlbchem_ctx* ctx);

/* Release ctx and its device memory (synchronises its last stream). NULL ok.
 * (Bookkeeping of the library; the paper has no counterpart.) */
void dlbchem_destroy(dlbchem_ctx* ctx);

/*
 * Host only, no GPU needed: build the mechanism tables for a team of
 * team_warps (1, 2, 4) warps and check them against the mechanism file, the
 * conditions the integrator's race-free gathers rely on (every incidence and
 * Jacobian entry exactly once with its coefficient, no target twice in a round
 * of 32, no target in two warps of one chunk, each target's entries in
 * reaction order). On success out[0..9] = chunks, reactions per chunk, D slots
 * per reaction, incidence rounds (all chunks and warps), Jacobian rounds,
 * whole-mechanism incidence rounds of the busiest warp, species split over two
 * accumulators, split offset, species, reactions. Returns OK, BAD_ARG or
 * BAD_MECH (message from dlbchem_last_error(NULL)).
 */
int dlbchem_table_stats(const char* mech_path, int32_t team_warps, int64_t* out);

/*
 * Host only, no GPU needed: a symbolic analysis of a sparse LU of the
 * iteration matrix I/(h gamma) - J (the problem-tailored linear algebra of
 * Sec. 5, future work), against the dense LU the integrator runs. The sparse
 * part of the species block is the pattern of d wdot_k / d c_j through the
 * reactions' own concentrations (participants, listed efficiencies) plus the
 * diagonal; the temperature row and column are dense, and the dense rank-1
 * term (the chain rule through rho and unit third-body efficiencies) is
 * taken by Sherman-Morrison. Species are eliminated by minimum degree on the
 * symmetrised pattern (ties to the lower index, no pivoting), temperature
 * last. On success out[0..9] = unknowns N, species-block nonzeros, L + U
 * nonzeros after fill (species pivots), dense LU multiply-adds, sparse LU
 * multiply-adds, dense and sparse multiply-adds of one pair of triangular
 * solves, the rank-1 extra per step, and the per-step totals (LU + four
 * solves) dense and sparse. Returns OK, BAD_ARG (NULL, more than 1024
 * species) or BAD_MECH.
 */
int dlbchem_lu_stats(const char* mech_path, int64_t* out);

#ifdef __cplusplus
}
#endif

#endif /* DLBCHEM_H */
