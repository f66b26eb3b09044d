/*
 * lelbm.h -- C ABI of the GB300 (sm_103a) implementation of the per-timestep
 * cell update of the Lagrangian entropic lattice Boltzmann method (LELBM),
 * W. Noh and C. Lee, arXiv:2508.06911.
 *
 * One time step ("lelbm_step") is, for every cell of a padded grid:
 *   - fluid boundary fill of the pad cells ............... Sec. III.A
 *   - macroscopic variables, non-equilibrium central moments,
 *     regularised central-moment collision, Knudsen limiter,
 *     normalisation (collision module, Fig. 6) ........... Eq. (IIB6)-(IIB18), App. C, App. D
 *   - Lagrangian acoustic stencil with internal refinement
 *     (LAS module, Fig. 7) .............................. Eq. (IIC6), (IIC9)-(IIC11)
 *   - entropic population reconstruction, Newton on the
 *     Lagrange multipliers with Cholesky solves (EPR module,
 *     Fig. 8) ........................................... Eq. (IID7)-(IID13)
 *   - moment streaming of T_N(c_i) rho f'_i and
 *     T_N(c_i) rho K RT g'_i to x + c_i (MS module, Fig. 9) Eq. (IIE3)
 * All quantities are in lattice units (dx = dt = dV = 1, Sec. II.A).
 *
 * State layout ("moments"): structure of arrays, [n_mom][n_cells] doubles, in
 * the order of Eq. (IIB5):
 *   1D: M0, Mx, Mxx, MDx, G0, Gx                              (n_mom = 6)
 *   2D: M0, Mx, My, Mxx, Mxy, Myy, MDx, MDy, G0, Gx, Gy       (n_mom = 11)
 *   3D: M0, Mx, My, Mz, Mxx, Mxy, Mxz, Myy, Myz, Mzz, MDx, MDy, MDz, G0, Gx,
 *       Gy, Gz                                                  (n_mom = 17)
 * where MD_g = sum_i |c_i|^2 c_ig f_i.  Cells run over the PADDED grid:
 *   2D: index = iy * NX + ix with NX = nx + 2 pad (nx if x is periodic),
 *       NY = ny + 2 pad (ny if y is periodic);
 *   3D: index = (iz * NY + iy) * NX + ix, NZ = nz + 2 pad (nz if z is
 *       periodic);
 *   1D: the instances of a batch are concatenated, each as
 *       [pad | interior of lengths[b] cells | pad] (no pads when periodic).
 * Pad cells are overwritten by the boundary fill at the start of every step;
 * after a step they read zero.
 *
 * Ownership: the library allocates and owns all device memory of a handle.
 * Host pointers passed in are read (or written) during the call only.
 * Functions ending in _device take device pointers the caller owns; they are
 * ordered on the handle's stream and do not synchronise.
 *
 * Errors: every function returns a status code.  The message of the last
 * failure of a handle is kept until the next failing call and is returned by
 * lelbm_last_error().  There is no CPU fallback: a handle cannot be created
 * without a CUDA device.
 */
#ifndef LELBM_H
#define LELBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LELBM_OK 0
#define LELBM_E_INVAL 1   /* invalid argument or parameter                   */
#define LELBM_E_NOMEM 2   /* device or host allocation failed                */
#define LELBM_E_CUDA 3    /* a CUDA call failed (message has the CUDA error)  */
#define LELBM_E_EPR 4     /* an EPR solve fell back to Maxwellian weights     */
#define LELBM_E_TIMEOUT 5 /* a bounded device wait ran out                    */
#define LELBM_E_STATE 6   /* non-physical state (rho <= 0, RT <= 0, NaN)      */

/* boundary kinds per side (x-, x+, y-, y+), Sec. III.A */
#define LELBM_BC_OUTFLOW 0  /* pads copy the nearest interior cell (zero gradient)   */
#define LELBM_BC_INFLOW 1   /* pads hold the equilibrium of the prescribed state      */
#define LELBM_BC_PERIODIC 2 /* wrap-around; must be set on both sides of an axis      */

/* arithmetic of the step */
#define LELBM_FP64 0  /* every operation in FP64                                     */
#define LELBM_MIXED 1 /* EPR Newton in FP32 to the FP32 noise floor, then per
                         population one Newton correction whose residual is summed
                         in double-float (FP32 pairs, about 48 bits) with an FP32
                         Jacobian, and a double-float streaming pass that re-checks
                         the residual of exactly the populations it deposits
                         against tol (a miss is taken back and corrected again,
                         then left to the FP64 EPR).  Exponents are exact int64
                         fixed-point polynomials, 2^w a table-driven double-float
                         exponential; deposits are FP64 atomic additions of both
                         words.  State, collision and accumulation in FP64.
                         Matches LELBM_FP64 to about 1e-13 per step.             */
#define LELBM_FP32 2  /* EPR Newton (passes and solves) and the streaming pass in
                         FP32, to an FP32 residual of 3e-4 (thermal units) plus one
                         polishing update; moment fractions widened to FP64 (exact
                         for normal numbers, subnormals dropped) and accumulated in
                         FP64; the emitted mass, momentum and energy are summed
                         exactly and their shortfall kept in the emitting cell, so
                         totals are conserved to FP64 rounding.  State, macroscopic
                         variables and non-equilibrium moments in FP64.  A cell
                         whose FP32 solve fails is solved by the FP64 EPR.  Error
                         against LELBM_FP64: about 1e-6 relative per step at
                         moderate temperatures, growing with the velocity set to
                         about 1e-4 at RT = 32 (q ~ 1700).  Over
                         thousands of 2D steps through the refinement switch
                         (RT = 4/9) the L1 density difference grows to about
                         1e-3, as it does for the FP64 scheme under noise of
                         that size.                                                 */

typedef struct lelbm* lelbm_t;

typedef struct {
    int dims;            /* 1, 2 or 3                                                  */
    int nx, ny;          /* interior cells (ny = 1 in 1D)                              */
    int n_batch;         /* 1D: number of independent instances (<= 1: a single one)   */
    const int* lengths;  /* 1D batch, host [n_batch]: interior length of each instance */
    const int* pads;     /* 1D batch, host [n_batch]: pad layers of each instance;
                            NULL: "pad" for every instance                           */
    int bc[4];           /* LELBM_BC_* for x-, x+, y-, y+                              */
    double inlet[4];     /* rho, ux, uy, RT of the inflow state                        */
    int pad;             /* pad layers on non-periodic sides (>= 1 if any)             */
    double K;            /* internal degrees of freedom, >= 0 (gamma = (D+K+2)/(D+K))  */
    double nu_shear;     /* kinematic shear viscosity, >= 0 (Eq. C8a)                  */
    double nu_bulk;      /* kinematic bulk viscosity (Eq. C8b); < 0 selects omega_b = 1 */
    double prandtl;      /* Prandtl number, > 0 (Eq. C8c)                              */
    int limiter;         /* 1: Knudsen limiter (App. D) on                              */
    double n_conform;    /* conformation number n of Eq. (IIC6); paper: 4              */
    double r_min;        /* minimum acoustic radius of Eq. (IIC6); paper: 2            */
    double refine_div;   /* divisor of N_r, Eq. (IIC9); paper: 3                       */
    double refine_rad;   /* refinement radius factor, Eq. (IIC10); paper: 3            */
    int max_refine;      /* cap on N_r, 0..4                                           */
    double tol;          /* EPR residual tolerance in thermal units; paper: 1e-12      */
    int max_newton;      /* Newton update cap per solve, 1..60                         */
    int precision;       /* LELBM_FP64, LELBM_MIXED or LELBM_FP32                      */
    const uint8_t* solid;/* host, one byte per padded cell: 0 fluid, 1 slip wall,
                            2 no-slip wall, 3 moving no-slip wall; NULL: none.  2D interior cells only
                            (flags on pads and in 1D are ignored).  Walls are
                            stationary and adiabatic (Sec. III.B).  A population
                            whose path crosses a solid face is specularly
                            reflected, exactly traced in 1/64-cell units.  Slip
                            walls: a cloud-in-cell share that would fall on a wall
                            cell is mirrored back across the wall.  No-slip walls
                            (FP64 path only): a population whose path touches one
                            is absorbed, with any share that would fall on one;
                            the cell then launches its own populations with -c_i
                            (the image populations of Eq. IIIB13 for u_w = 0) and
                            those whose paths touch the wall enter, scaled to the
                            absorbed mass (Eq. IIIB14-IIIB15).  3: a no-slip wall
                            moving at wall_u (tangentially; the cell stays solid):
                            its images are the EPR populations of the cell's
                            post-collision central constraints at the bulk
                            velocity u - 2 u_w (Eq. IIIB10-IIIB11).  An outflow pad
                            whose nearest interior cell is a wall is that wall.  */
    void* stream;        /* cudaStream_t to run on; NULL: a stream owned by the handle  */
    /* three dimensions (dims = 3; ignored below).  FP64 path with the Eq. (IID13)
       start, fluid boundaries only (no solid cells, warm-start store or network,
       batches).  One warp updates one cell; its velocity set is laid out as at
       most 1024 runs of points along x (R_ac up to about 16, RT up to about 16
       at the paper's n = 4).  A cell whose set does not fit is not streamed and
       is counted as a Maxwellian fallback (lelbm_synchronize: E_EPR). */
    int nz;              /* interior cells along z                                      */
    int bc_z[2];         /* LELBM_BC_* for z-, z+                                       */
    double inlet_uz;     /* z velocity of the inflow state (inlet[] holds rho, ux, uy, RT) */
    int deterministic;   /* 1: moment streaming as a gather in a fixed order instead of
                            FP64 atomic scatters, so repeated runs give the same bits
                            whatever else the GPU runs (2D, LELBM_FP64, no solid cells;
                            E_INVAL otherwise).  The cell kernel keeps each cell's
                            multipliers ((N_f + N_g) doubles per cell, 128 B in 2D) for
                            a gather kernel in which every target cell sums what the
                            cells within reach send it (Eq. IIE3).                    */
    double wall_u[2];    /* velocity u_w of the moving no-slip walls (solid byte 3),
                            Eq. (IIIB2)-(IIIB4)                                        */
} lelbm_params;

/* Per-handle counters accumulated by every step since the last reset. */
typedef struct {
    long long steps;              /* time steps taken                               */
    long long cells;              /* cell updates (emitting cells x steps)          */
    long long newton_hist[64];    /* Newton updates per solve, f and g solves alike */
    long long fallback_eq;        /* cells re-solved with equilibrium constraints   */
    long long fallback_mx;        /* cells given normalised Maxwellian weights      */
    long long q_max;              /* largest velocity set                           */
    double disp_max;              /* largest |c_i| streamed (lattice Courant, IIC3) */
    long long first_fail_cell;    /* first cell with a Maxwellian fallback, or -1   */
    double cell_kernel_ms;        /* CUDA-event time of the cell-update kernel      */
    long long cell_kernel_launches;/* launches timed into cell_kernel_ms            */
    long long points_f;           /* stencil points visited by fluon Newton passes  */
    long long points_g;           /* stencil points visited by phonon Newton passes */
    long long points_ms;          /* stencil points streamed (moment streaming)     */
    long long points_32;          /* stencil points of FP32 Newton passes           */
    long long judge_redo;         /* mixed: cells re-solved in FP64 after the check;
                                     FP32: cells whose FP32 solve failed (FP64 EPR) */
    long long mlp_retry;          /* learned or stored start failed; re-solved from
                                     Eq. (IID13)                                    */
    long long wall_hits;          /* populations specularly reflected at a solid
                                     face while streaming (Sec. III.B)              */
    long long mlp_cells;          /* cells given the learned warm start             */
    long long points_df;          /* mixed: stencil points of double-float streaming
                                     passes (deposits and take-backs)               */
    long long points_df_corr;     /* mixed: stencil points of double-float Newton
                                     correction passes                              */
} lelbm_stats;

/* Sizes of the structures this library was built with, so a binding can check
 * its own layout: sizeof(lelbm_params), sizeof(lelbm_stats). */
void lelbm_abi_sizes(long long* params_size, long long* stats_size);

/* Fill p with the paper's defaults (n = 4, R_min = 2, refinement 3/3, tol 1e-12,
 * limiter on, omega_b = 1, Pr = 1, K = 0) for a 1D grid of 1 cell, every axis periodic
 * (x, y and z, so that setting dims and the sizes alone gives a fully periodic grid). */
void lelbm_default_params(lelbm_params* p);

/* Validate p, allocate the device state (two moment buffers, cell types, the
 * instance table, counters) and return a handle in *out.  The state starts at
 * zero; set it with lelbm_set_state or lelbm_set_moments.  The host arrays
 * p->lengths, p->pads and p->solid are read during the call only; the handle keeps
 * no pointer to them or to p.  The parameters are validated before any CUDA call,
 * so an invalid set gives E_INVAL (with the reason in lelbm_last_error(NULL)) also
 * on a machine without a GPU.
 * Errors: E_INVAL (bad parameter), E_NOMEM, E_CUDA (no device). */
int lelbm_create(lelbm_t* out, const lelbm_params* p);

/* Release the handle and its device memory.  NULL is ignored. */
void lelbm_destroy(lelbm_t h);

/* Sizes of the padded state: total cells, moments per cell, NX, NY (1D: NX =
 * total concatenated cells, NY = 1).  Any output pointer may be NULL. */
int lelbm_layout(lelbm_t h, long long* n_cells, int* n_mom, int* NX, int* NY);

/* Interior cell range of 1D instance b: first interior cell and length. */
int lelbm_instance(lelbm_t h, int b, long long* first, int* length);

/* Equilibrium moments (Eq. IIB7) from host primitive fields over the padded
 * grid: rho[n_cells], u[dims][n_cells] (SoA), RT[n_cells].  Pad and solid
 * cells are ignored.  Errors: E_STATE if an interior fluid cell has
 * rho <= 0, RT <= 0 or a non-finite value. */
int lelbm_set_state(lelbm_t h, const double* rho, const double* u, const double* RT);

/* Copy a host moment state [n_mom][n_cells] in (checkpoint restore). */
int lelbm_set_moments(lelbm_t h, const double* m);

/* Same from a device buffer owned by the caller (asynchronous on the stream). */
int lelbm_set_moments_device(lelbm_t h, const double* m_dev);

/* Enqueue n time steps on the handle's stream (n >= 0).  Returns after the
 * launches; errors of the launches themselves are reported here, counters
 * and EPR fallbacks at the next synchronising call. */
int lelbm_step(lelbm_t h, int n);

/* Wait for the stream.  Returns E_EPR if a cell needed the Maxwellian
 * fallback since the last reset of the counters, E_CUDA on a device error. */
int lelbm_synchronize(lelbm_t h);

/* Copy the current moment state to a host buffer [n_mom][n_cells]; syncs. */
int lelbm_get_moments(lelbm_t h, double* m);

/* Copy the current moment state to a caller-owned device buffer (async). */
int lelbm_get_moments_device(lelbm_t h, double* m_dev);

/* Macroscopic fields (Eq. IIB6) to host buffers rho[n_cells],
 * u[dims][n_cells], RT[n_cells]; pads and solid cells read zero; syncs. */
int lelbm_get_macros(lelbm_t h, double* rho, double* u, double* RT);

/* Counters since the last reset; syncs. */
int lelbm_get_stats(lelbm_t h, lelbm_stats* s);

/* Zero the counters. */
int lelbm_reset_stats(lelbm_t h);

/* 1: time every cell-update kernel with CUDA events on its own stream. */
int lelbm_set_timing(lelbm_t h, int on);

/* ---- 1D batches: persistent execution ----------------------------------
 * Per-instance step budgets for lelbm_run_batch (host array [n_batch]; NULL
 * removes every budget).  An instance whose budget is spent is frozen. */
int lelbm_set_steps(lelbm_t h, const int* steps);

/* Launch shape of the persistent batch kernel. */
typedef struct {
    int threads;        /* threads per block: 64 or 128                          */
    int blocks_per_sm;  /* resident blocks per SM (0: the occupancy maximum)     */
    int order;          /* 0: instances in batch order, 1: longest first         */
    double ms;          /* autotune: time of the trial, else 0                   */
} lelbm_tuning;

/* Advance every 1D instance by min(n, its budget) time steps in ONE persistent
 * kernel launch, replayed from a CUDA graph captured on the first call with
 * this n.  A block claims a whole instance and runs its steps with block-level
 * barriers (instances share no cells); results equal n calls of lelbm_step
 * when no budget is set.  1D handles only (E_INVAL otherwise); asynchronous. */
int lelbm_run_batch(lelbm_t h, int n);

/* Time every candidate launch shape (threads 64/128, 1, 2 or the maximum of
 * blocks per SM, batch or longest-first order) for trial_steps steps on the
 * current state, restore the state and budgets after each trial, keep the
 * fastest for lelbm_run_batch and return it in *best (may be NULL).  Syncs. */
int lelbm_autotune(lelbm_t h, int trial_steps, lelbm_tuning* best);

/* Set the launch shape of lelbm_run_batch explicitly. */
int lelbm_set_tuning(lelbm_t h, const lelbm_tuning* t);

/* ---- Learned warm start of the EPR Newton -----------------------------------
 * The Newton of Sec. II.D starts from the Maxwellian multipliers of Eq. (IID13);
 * with a network set, it starts from those plus a correction predicted by an MLP
 * (2 x 64 hidden units, SiLU, BF16 weights, FP32 accumulation) from the cell's
 * normalised post-collision constraints and stencil geometry.  The plain start
 * stays the fallback (a failed learned solve is redone from Eq. IID13) and the
 * same residual tolerance is the judge, so results do not depend on the network.
 * Features: 8 (1D) / 15 (2D); targets: converged multipliers minus Eq. (IID13)
 * in thermal units, fluons then phonons, 7 (1D) / 16 (2D).  Parameters: FP32
 * vector W1 b1 W2 b2 W3 b3 followed by the input/output means and standard
 * deviations (n_params in total, the first n_weights trained). */
int lelbm_mlp_size(int dims, int* n_in, int* n_out, long long* n_params, long long* n_weights);

/* Initial parameters into the HOST array params[n_params]: He-uniform weights
 * (seeded) and the normalisation from n training pairs X_dev[n][n_in],
 * Y_dev[n][n_out] on the device (n = 0: unit normalisation).  Syncs. */
int lelbm_mlp_init(int dims, unsigned long long seed, const float* X_dev, const float* Y_dev, long long n,
                   float* params);

/* Mean-squared loss (standardised targets) and its gradient with respect to the
 * n_weights trained parameters, at the BF16-rounded weights, over all n pairs;
 * params_dev, X_dev, Y_dev, grad_dev are device arrays; *loss is host.  Syncs. */
int lelbm_mlp_loss_grad(int dims, const float* params_dev, const float* X_dev, const float* Y_dev, long long n,
                        float* grad_dev, double* loss, void* stream);

/* Train params_dev in place: epochs of shuffled minibatches, Adam (lr, beta
 * 0.9/0.999) on FP32 master weights, BF16 forward/backward with FP32
 * accumulation.  epoch_loss (host, may be NULL) gets the mean loss of each epoch. */
int lelbm_mlp_train(int dims, float* params_dev, const float* X_dev, const float* Y_dev, long long n, int epochs,
                    int batch, float lr, unsigned long long seed, double* epoch_loss, void* stream);

/* One time step that also writes, for every cell solved without fallback, its
 * features to x_dev[cell][n_in] and its targets to y_dev[cell][n_out] (device
 * arrays over the padded cells; other rows are left untouched). */
int lelbm_step_record(lelbm_t h, float* x_dev, float* y_dev);

/* The warm-start network's inference as lelbm_step runs it (BF16 weights and BF16
 * activations between the layers on the tensor cores, FP32 accumulation, SiLU in FP32
 * rounded to BF16; the persistent batch of lelbm_run_batch uses the packed BF16 tanh
 * for SiLU instead) on n caller-supplied feature rows: X_dev[n][n_in] (device) ->
 * Y_dev[n][n_out] (device, predicted targets in raw units).  params: host, n_params
 * floats, as for lelbm_set_mlp.  Allocates two small device buffers; syncs the stream
 * (NULL: the legacy default stream).  Errors: E_INVAL, E_NOMEM, E_CUDA. */
int lelbm_mlp_infer(int dims, const float* params, const float* X_dev, long long n, float* Y_dev, void* stream);

/* Use the network params (host, n_params floats) as warm start; NULL: the plain
 * Maxwellian start. */
int lelbm_set_mlp(lelbm_t h, const float* params);

/* Gate of the learned start: a cell whose normalised post-collision constraints
 * (thermal units, Eq. IIB16-IIB18) all lie within `departure` of their
 * equilibrium values (1, 0, delta_ab, 0 for fluons; 1, 0 for the phonons' free
 * ones) starts from Eq. (IID13) instead of the network: near equilibrium
 * Eq. (IID13) is closer to the solution than the network's fit.  A warp whose 32
 * cells are all gated out skips the network.  0 (the default) uses the network
 * for every cell.  Applies to the learned start of the cell-update path (not the
 * persistent 1D batch).  Errors: E_INVAL (departure < 0 or not finite), E_CUDA. */
int lelbm_set_mlp_gate(lelbm_t h, double departure);

/* Stored warm start (Sec. II.D: the multipliers of each cell kept as the
 * precondition of its next step).  stored = 1 allocates a per-cell FP32 store of
 * the converged multipliers minus Eq. (IID13) ((N_f + N_g) floats per cell: 7 in
 * 1D, 16 in 2D; zero at first, so the first step starts from Eq. IID13).  Every
 * solve then starts from Eq. (IID13) plus the cell's stored correction and writes
 * the new one.  A start that does not converge is retried from Eq. (IID13)
 * (counted in mlp_retry); a cell solved by a fallback stores zero.  Where the
 * learned start is set, it takes precedence.  stored = 0 frees the store.
 * Errors: E_NOMEM, E_CUDA. */
int lelbm_set_warmstart(lelbm_t h, int stored);

/* Measured FMA throughput of the current device in FLOP/s (2 per FMA), FP32 pipe
 * (fp64 = 0) or FP64 pipe (fp64 = 1): a probe kernel of eight independent FMA
 * chains per thread on 8 blocks of 256 threads per SM, best of three timed launches
 * after a warm-up (about 0.1 s).  It is the denominator of the ALU rooflines the
 * benchmark reports; the paper has no counterpart.  Syncs the device.
 * Errors: E_INVAL (flops NULL), E_CUDA. */
int lelbm_fma_peak(int fp64, double* flops);

/* Checks of the mixed path's double-float building blocks on caller data (host
 * arrays, copied in and out; the call allocates device memory and syncs the
 * device).  The paper has no counterpart: they let a test hold the FP32-pipe
 * arithmetic of LELBM_MIXED against FP64.
 * lelbm_df_exp2: out[i] = 2^(w[i] 2^-54) by the table-driven double-float
 *   exponential of the mixed path's EPR passes (Tang's method), as FP64;
 *   w[i] in [-120, 200] 2^54.
 * lelbm_df_dot: out[r] = sum_t k[r*n_terms + t] v[r*n_terms + t], each v split
 *   into a double-float and accumulated in the double-float accumulator of the
 *   streaming and correction passes, in index order, one row per thread.
 * Errors: E_INVAL (sizes, NULL, w out of range), E_NOMEM, E_CUDA. */
int lelbm_df_exp2(const long long* w, long long n, double* out);
int lelbm_df_dot(const float* k, const double* v, long long n_terms, long long n_rows, double* out);

/* Message of the last failure of h ("" if none; h may be NULL for create). */
const char* lelbm_last_error(lelbm_t h);

/* ---- Allocation-free single step (the paper has no counterpart) ----------
 * For callers that must not allocate device memory: an application that owns all
 * device memory through its own pool or a fixed budget, or code on a latency-
 * critical path where cudaFree synchronises the device and cudaMalloc can fail or
 * fragment.  The caller passes the state buffers it already owns; the step itself
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * p:      the parameters of lelbm_create for a 1D or 2D grid, with solid == NULL,
 *         precision FP64, deterministic == 0 and at most
 *         LELBM_NOALLOC_MAX_INSTANCES 1D instances; p->stream is the
 *         stream to run on (NULL: the legacy default stream).
 * m_in:   device [n_mom][n_cells] moments at time t in the padded layout above;
 *         pad cells are not read (they are derived from the interior or the
 *         inflow state); not modified.
 * m_out:  device [n_mom][n_cells], overwritten with the moments at t + 1 (pad
 *         cells zero).  Must not overlap m_in.
 * stats:  NULL: return after enqueueing the work (asynchronous).  Otherwise the
 *         call waits for the stream and fills *stats for this step.
 * Returns E_INVAL (bad parameter or more instances than the maximum), E_CUDA, or
 * E_EPR (only with stats != NULL) when a cell fell back to Maxwellian weights.
 *
 * Scratch: a file-scope device array of 512 KiB (counters and the instance table),
 * held by every GPU on which the library is loaded until the process exits.  The
 * first call on a device looks up the array's device address; make that first
 * call before any stream capture.  All calls share the array and each call resets
 * what it reads, so calls whose work overlaps on the GPU race with each other. */
#define LELBM_NOALLOC_MAX_INSTANCES 16384
int lelbm_step_noalloc(const lelbm_params* p, const double* m_in, double* m_out, lelbm_stats* stats);

#ifdef __cplusplus
}
#endif

#endif /* LELBM_H */
