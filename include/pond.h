/*
 * pond.h -- C ABI of the GB300 (sm_103a) library for the regularized Particles-on-Demand
 * finite-volume scheme of Kallikounis, Dorschner and Karlin, "Particles on Demand for
 * flows with strong discontinuities" (arXiv 2203.05477).
 *
 * One time step (Sec. III.B.4) re-expresses every cell in its co-moving frame
 * (Sec. II.C), evaluates the face populations at t_{n+1/2} by the face predictor-
 * corrector (Sec. III.B.3), forms the fluxes Eq. (fluxEq) in each cell's frame and
 * applies the co-moving DUGKS update Eqs. (FinalUpdateDUGKS).  All of it runs in CUDA
 * kernels on the device; the host only launches them.
 *
 * Conventions
 *   - Every call returns a pond_status; nothing else crosses the ABI (no exceptions).
 *   - Host arrays are plain C arrays; device arrays are CUDA device pointers.  Fields are
 *     structure-of-arrays of nx*ny FP64 values, x fastest.
 *   - The library owns a pond_state and everything it allocates; the caller owns every
 *     array it passes in.  Device memory comes from the allocator in pond_options (for
 *     example the caller's caching allocator) or, when that is NULL, from cudaMalloc.
 *   - All work is enqueued on the stream given in pond_options (NULL: the library creates
 *     and owns a non-blocking stream).  One state is used by one stream at a time.
 *   - Device-side conditions (a non-physical state, a face whose corrector found no
 *     frame) are sticky: they are recorded on the device and reported by pond_sync.
 *   - Thread safety: distinct states may be used from distinct threads.  The message of
 *     pond_last_error is thread-local.
 */
#ifndef POND_H
#define POND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    POND_OK = 0,
    POND_ERR_INVALID_ARG = 1,    /* a NULL pointer, a size <= 0, a bad enum value */
    POND_ERR_UNSUPPORTED = 2,    /* velocity set other than D1Q4/D2Q16; gamma > 1 + 2/D */
    POND_ERR_OOM = 3,            /* the allocator returned NULL */
    POND_ERR_CUDA = 4,           /* a CUDA runtime call failed; see pond_last_error */
    POND_ERR_NONPHYSICAL = 5,    /* rho <= 0, T <= 0 or not finite in a cell, or a face whose
                                    corrector found no frame (reported by pond_sync) */
    POND_ERR_NOT_CONVERGED = 6,  /* reported by pond_sync when strict_convergence is set */
    POND_ERR_TIMEOUT = 7         /* a bounded device-side wait gave up */
} pond_status;

/* Velocity sets of Table I: D1Q4 (Gauss-Hermite roots of He_4, T_L = 1) and its tensor
 * product D2Q16 (Eq. wi).  D1Q3/D2Q9 cannot carry the third-order Grad projection the
 * paper requires (Sec. II.C) and are refused with POND_ERR_UNSUPPORTED.  D3Q64, the tensor
 * product in three dimensions, is created by pond_init3 (pond_init refuses it). */
typedef enum { POND_D1Q3 = 0, POND_D1Q4 = 1, POND_D2Q16 = 2, POND_D2Q9 = 3, POND_D3Q64 = 4 } pond_velset;

/* Ghost-cell rules (two layers): copy of the nearest cell (zero gradient), wrap-around,
 * the equilibrium at a prescribed state on part of a side (transmissive on the rest), or a
 * reflective wall: ghost k mirrors the k-th cell from the wall, with the normal component
 * of every particle velocity and of the frame velocity reversed (the two-blast-wave and
 * explosion-in-a-box cases of Sec. IV). */
typedef enum { POND_BC_TRANSMISSIVE = 0, POND_BC_PERIODIC = 1, POND_BC_INFLOW = 2, POND_BC_REFLECTIVE = 3 } pond_bc;

/* Arithmetic of populations, fluxes and collision.  Frames (u, T) advance by increments
 * formed relative to the old frame; they are FP64 words in FP64 mode and float-float pairs
 * (about 48 significant bits) in FP32 mode. */
typedef enum { POND_FP64 = 0, POND_FP32 = 1 } pond_precision;

/* Slope limiters named in Sec. III.B.3: van Leer and minmod. */
typedef enum { POND_VANLEER = 0, POND_MINMOD = 1 } pond_limiter;

typedef struct {
    int dim;                    /* 1 or 2; must match the velocity set */
    int64_t nx, ny;             /* cells; ny is ignored (taken as 1) when dim == 1 */
    double x0, x1, y0, y1;      /* domain [x0,x1] x [y0,y1]; cell centres at (k + 1/2) dx */
    int bc[4];                  /* pond_bc for sides x-lo, x-hi, y-lo, y-hi */
    double inflow[4][4];        /* per side: rho, ux, uy, p of the inflow state */
    int64_t inflow_lo[4];       /* inflow applies to cells [lo, hi) along that side */
    int64_t inflow_hi[4];
} pond_grid;

/* Time-stepping realizations of Sec. III: the finite-volume scheme (Sec. III.B, the
 * conservative default) or the semi-Lagrangian one (Sec. III.A: per-node predictor-
 * corrector on the node's frame, populations advected from their departure points by a
 * limited 4-point Lagrange interpolation, in 2D its limited tensor product, BGK
 * collision; not conservative).  The semi-Lagrangian scheme runs on D1Q4 and D2Q16 grids;
 * batches refuse it with POND_ERR_UNSUPPORTED, and it keeps no face frames
 * (pond_face_gauges returns POND_ERR_UNSUPPORTED). */
typedef enum { POND_FV = 0, POND_SL = 1 } pond_scheme;

typedef struct {
    int precision;              /* pond_precision */
    int limiter;                /* pond_limiter */
    double cfl;                 /* CFL = max|v_ia| dt / dx (Sec. IV); e.g. 0.2 */
    double t_end;               /* > 0: the last step is clipped to t_end, later ones are no-ops */
    double tol;                 /* corrector stop: |du| <= tol sqrt(T) and |dT| <= tol T */
    int max_iter;               /* corrector passes at most (e.g. 16) */
    int fixed_iters;            /* > 0: exactly this many passes per face (parity mode) */
    int strict_convergence;     /* nonzero: faces that hit max_iter make pond_sync fail */
    int learned;                /* nonzero: the learned face-gauge predictor seeds the corrector */
    void *stream;               /* cudaStream_t, or NULL for a stream the library creates */
    void *(*alloc)(size_t bytes, void *ctx);  /* device allocator, or NULL for cudaMalloc */
    void (*free)(void *ptr, void *ctx);
    void *alloc_ctx;
    int scheme;                 /* pond_scheme (0: finite volume) */
} pond_options;

typedef struct pond_state pond_state;

/* Diagnostics gathered on the device since pond_init / pond_set_primitive. */
typedef struct {
    double t;                   /* simulated time */
    double dt;                  /* time step of the next step */
    int64_t steps;              /* steps taken */
    int64_t face_solves;        /* faces processed (faces x steps) */
    int64_t face_iters;         /* corrector passes summed over all faces */
    int64_t nonconverged;       /* faces that stopped at max_iter */
    int64_t fallbacks;          /* passes that defined no frame (restart / stop early) */
    int64_t nonphysical;        /* non-physical cells or faces */
    int64_t first_bad_cell;     /* index of the first non-physical cell, or -1 */
    uint32_t flags;             /* bit 0 non-physical, bit 1 not converged, bit 2 timeout */
    int64_t staged_tma;         /* face-kernel tiles whose box was staged by tensor-map (TMA)
                                   copies (the TMA variant of the D2Q16 FP32 face kernel) */
} pond_diag;

/* Creates a solver for the problem statement of the paper's benchmarks (Sec. IV): grid and
 * boundary conditions, velocity set, ratio of specific heats gamma (Cv = 1/(gamma-1),
 * p = rho T), BGK relaxation time tau (Eqs. f_equation, g_equation).  gamma must satisfy
 * Cv >= D/2 (Eq. geqPond), i.e. gamma <= 1 + 2/D.  Allocates all device memory once. */
pond_status pond_init(const pond_grid *grid, pond_velset velset, double gamma, double tau,
                      const pond_options *opts, pond_state **out);

/* Three-dimensional grids (D3Q64: W_i = w_ix w_iy w_iz of the D1Q4 rule; the extension the
 * paper names as future work in Sec. V, with the 20 slow f moments of Sec. II.C for D = 3).
 * Box [x0,x1] x [y0,y1] x [z0,z1] of nx x ny x nz cells; fields are nx*ny*nz values, x
 * fastest, then y.  Sides are transmissive, periodic (in pairs) or reflective; no inflow. */
typedef struct {
    int64_t nx, ny, nz;
    double x0, x1, y0, y1, z0, z1;
    int bc[6];                  /* pond_bc for sides x-lo, x-hi, y-lo, y-hi, z-lo, z-hi */
} pond_grid3;

/* pond_init for a D3Q64 grid: the finite-volume scheme (Sec. III.B) with the face
 * corrector of Sec. III.B.3 on the faces of all three axes (two tangential limited slopes
 * per face).  gamma <= 5/3 (Cv >= 3/2, Eq. geqPond).  The learned predictor and the
 * semi-Lagrangian scheme are D1Q4/D2Q16 features: options asking for them are refused
 * with POND_ERR_UNSUPPORTED.  On the returned state pond_step, pond_step_timed,
 * pond_sync, pond_get_state (coef_f [cells][20], coef_g [cells][10], frame [cells][4]:
 * ux, uy, uz, T; coefficient (r, s, t) at position (r+s+t)(r+s+t+1)(r+s+t+2)/6 +
 * (s+t)(s+t+1)/2 + t) and pond_destroy work as for the other grids; initial conditions,
 * moments and face frames go through the three calls below. */
pond_status pond_init3(const pond_grid3 *grid, double gamma, double tau, const pond_options *opts, pond_state **out);
/* pond_set_primitive with the third velocity component uz (all five fields required). */
pond_status pond_set_primitive3(pond_state *s, const double *rho, const double *ux, const double *uy,
                                const double *uz, const double *p, int on_device);
/* pond_moments with the third momentum component; totals[5] (rho, mx, my, mz, E). */
pond_status pond_moments3(pond_state *s, double *rho, double *mx, double *my, double *mz, double *E,
                          double totals[5], int on_device);
/* Face frames of the three axes, [nf][4] (ux, uy, uz, T) each: x-faces (nx+1)*ny*nz,
 * y-faces nx*(ny+1)*nz, z-faces nx*ny*(nz+1), x fastest.  NULL arrays are skipped. */
pond_status pond_get_face_gauges3(pond_state *s, double *xg, double *yg, double *zg);
pond_status pond_set_face_gauges3(pond_state *s, const double *xg, const double *yg, const double *zg);

/* Initial condition: the co-moving equilibria Eqs. (feqPond), (geqPond) of primitive
 * fields rho, ux, uy, p (uy may be NULL in 1D).  on_device: the arrays are device
 * pointers (else host).  Also sets the face predictors (the frame of the pooled moments
 * of the two adjacent cells), t = 0 and the first time step. */
pond_status pond_set_primitive(pond_state *s, const double *rho, const double *ux,
                               const double *uy, const double *p, int on_device);

/* Enqueues n_steps time steps (Sec. III.B.4) on the state's stream and returns without
 * waiting.  The time step of each step comes from the CFL condition on the device. */
pond_status pond_step(pond_state *s, int64_t n_steps);

/* Same as pond_step, but launches every kernel individually with CUDA events around it on
 * the state's stream, waits, and adds the elapsed milliseconds of all face-corrector
 * launches to ms[0] and of all cell-update launches to ms[1] (ms: host array of 2). */
pond_status pond_step_timed(pond_state *s, int64_t n_steps, double ms[2]);

/* Conserved fields rho, rho ux, rho uy, rho E per cell (Sec. II.B) into caller buffers
 * (host or device per on_device; any pointer may be NULL to skip it) and, if totals is
 * not NULL, their compensated FP64 sums over the grid times the cell volume.  Waits for
 * the stream. */
pond_status pond_moments(pond_state *s, double *rho, double *mx, double *my, double *E,
                         double totals[4], int on_device);

/* The stored state for inspection: per cell its Hermite coefficients in its own frame
 * (D1Q4: f a0..a3, g b0..b2; D2Q16: f a00,a10,a01,a20,a11,a02,a30,a21,a12,a03 and g
 * b00,b10,b01,b20,b11,b02; [cells][ncoef]) and frame (u..., T) ([cells][D+1]).  Host
 * buffers; waits for the stream.  coef_f/coef_g/frame may be NULL. */
pond_status pond_get_state(pond_state *s, double *coef_f, double *coef_g, double *frame);

/* Face predictors (u..., T) for x-faces [(nx+1)*ny][D+1] and (2D) y-faces
 * [nx*(ny+1)][D+1]; host buffers.  pond_set_face_gauges overwrites them. */
pond_status pond_get_face_gauges(pond_state *s, double *xg, double *yg);
pond_status pond_set_face_gauges(pond_state *s, const double *xg, const double *yg);

/* Batched 1D shock tubes (D1Q4): n_tubes independent tubes, tube k with lengths[k] cells
 * of width dx[k] (NULL: 1/lengths[k], i.e. every tube spans [0, 1]) and ratio of specific
 * heats gammas[k], transmissive ends, one relaxation time tau.  Each tube keeps its own
 * time and CFL time step.  The other calls take concatenated arrays (tube after tube, x
 * fastest): pond_set_primitive (uy NULL), pond_moments (my left zero; totals summed over
 * tubes), pond_get_state, pond_get_face_gauges (tube k has lengths[k] + 1 faces).
 * pond_step(n) advances every tube by n of its own steps in one persistent kernel launch
 * (one CTA per tube, no inter-CTA synchronization).  Used for the batched-tube workload of
 * the paper's 1D benchmarks (Sec. IV.A-IV.B). */
pond_status pond_init_batch(int64_t n_tubes, const int64_t *lengths, const double *gammas, const double *dx,
                            double tau, const pond_options *opts, pond_state **out);

/* Per-tube simulated time t[k] and next time step dt[k] of a batch (host arrays, may be
 * NULL); waits for the stream. */
pond_status pond_batch_times(pond_state *s, double *t, double *dt);

/* Per-tube status of a batch (0 running, 1 stopped: the tube reached a non-physical state
 * and is no longer advanced) and the number of steps each tube has taken (host arrays,
 * may be NULL); waits for the stream. */
pond_status pond_batch_status(pond_state *s, int32_t *status, int64_t *steps_done);

/* ---- Learned face-gauge predictor (D2Q16 grids).  Not part of the paper: a small MLP
 * (48 -> 64 -> 64 -> 3, BF16 tensor-core GEMMs with FP32 accumulation) predicts each face's
 * converged corrector frame from its stencil, and the prediction replaces the previous
 * half step's frame as the corrector's starting point.  The corrector and its convergence
 * test are unchanged.  Parameters: POND_MLP_PARAMS FP32 values laid out
 * W1[64][48] b1[64] W2[64][64] b2[64] W3[16][64] b3[16]; a new state starts from seeded
 * random W1, W2 and zero W3, b (prediction = the previous frame). */
#define POND_MLP_PARAMS 8336
#define POND_MLP_FEATURES 48
#define POND_MLP_PAIR_STRIDE 52   /* a training pair: 48 features, 3 targets, the face's corrector passes */

/* Runs n_steps plain steps and samples (features, converged face frame) pairs from every
 * every-th converged face into pairs (device, [cap][POND_MLP_PAIR_STRIDE] floats); the
 * number written (at most cap) goes to *n_out. */
pond_status pond_gauge_collect(pond_state *s, int64_t n_steps, float *pairs, int64_t cap, int every, int64_t *n_out);

/* Trains the state's network on n pairs (device) with Adam (learning rate lr) and mean
 * squared error, in minibatches of `batch` consecutive pairs (the caller shuffles), for
 * `epochs` epochs; loss_out (host, may be NULL) receives the mean loss of each epoch. */
pond_status pond_gauge_train(pond_state *s, const float *pairs, int64_t n, int epochs, int batch, float lr,
                             float *loss_out);

/* Switches the learned predictor on (nonzero) or off for the following steps.  The face
 * corrector starts from the prediction where the largest component of the predicted
 * (normalized) correction exceeds `gate` (default 0.01) and does not exceed `trust`
 * (default 0.5: larger moves can lead the corrector to another fixed point).  It keeps the
 * result only if it converges without a restart; otherwise it solves the face again from
 * the previous half step's frame, as without the network, so the corrector alone decides
 * the result.
 * Errors: INVALID_ARG for gate < 0 or trust <= 0. */
pond_status pond_gauge_enable(pond_state *s, int on);
pond_status pond_gauge_set_gate(pond_state *s, float gate);
pond_status pond_gauge_set_trust(pond_state *s, float trust);

/* The equilibration alternative of Sec. II.C, as an ablation of Grad's projection (the
 * paper's choice, and the default): with on nonzero, every change of frame of the
 * following steps keeps the slow moments (third order for f, second for g) and sets the
 * fast tensor-Hermite components He_r(c_x) He_s(c_y) (r, s <= 3 beyond those orders) to
 * the values of the equilibrium with the population's own zeroth and first moments in the
 * new frame.  One kernel tile is compiled for it, so pond_autotune has nothing to choose.
 * Errors: UNSUPPORTED on batches, D3Q64 grids, the semi-Lagrangian scheme, or with the
 * learned predictor on. */
pond_status pond_set_equilibration(pond_state *s, int on);

/* The network as a self-describing byte blob (magic, version, count, parameters) for
 * checkpointing: pond_gauge_save writes it to buf (host) if *size is large enough and
 * always sets *size to the bytes needed; pond_gauge_load reads one back. */
pond_status pond_gauge_save(pond_state *s, void *buf, size_t *size);
pond_status pond_gauge_load(pond_state *s, const void *buf, size_t size);

/* Copies the network parameters from / to host arrays of POND_MLP_PARAMS floats. */
pond_status pond_gauge_set_params(pond_state *s, const float *params);
pond_status pond_gauge_get_params(pond_state *s, float *params);

/* Stand-alone network calls on device arrays, enqueued on `stream` (NULL: legacy default
 * stream) and waited for: forward pass of n rows x[n][ldx] (first 48 columns) into
 * out[n][16]; and the gradient of the mean squared error against the targets held in
 * columns 48..50 of y[n][ldy] into grad[POND_MLP_PARAMS] and the loss into *loss (device
 * floats).  pond_mlp_gradient allocates its activation scratch with cudaMalloc. */
pond_status pond_mlp_forward(const float *params, const float *x, int ldx, int64_t n, float *out, void *stream);
pond_status pond_mlp_gradient(const float *params, const float *x, int ldx, const float *y, int ldy, int64_t n,
                              float *grad, float *loss, void *stream);

/* pond_mlp_gradient without any device allocation.  The paper has no counterpart: this is
 * a service for callers that cannot call cudaMalloc, for example code running while a
 * framework's caching allocator has reserved the whole device, code that must not add the
 * device-wide synchronization cudaMalloc/cudaFree imply, or code on a path where a failed
 * allocation cannot be handled.  Inputs and outputs are as for pond_mlp_gradient (device
 * arrays owned by the caller).  The activation scratch lives in a fixed device array of
 * the library sized for POND_MLP_NOALLOC_MAX_ROWS rows (about 6.6 MB, held by every GPU that
 * loads the library until the process exits); n above that limit returns
 * POND_ERR_INVALID_ARG.  Every call looks up that array's device address in the current
 * context (no allocation); the first call on a device also sets the kernels' shared-memory
 * limit for that device and loads the array's module, so make the first call before any
 * stream capture.  All calls share the one array: calls whose work overlaps on the GPU
 * (different streams, or threads calling concurrently) race on it; serialize them.  The
 * call clears *loss and its error word itself, enqueues on `stream`, and waits for it.
 * On POND_ERR_TIMEOUT grad is left as it was (the weight-gradient kernel does not run on
 * incomplete activations) and *loss is undefined. */
#define POND_MLP_NOALLOC_MAX_ROWS 8192
pond_status pond_mlp_gradient_noalloc(const float *params, const float *x, int ldx, const float *y, int ldy, int64_t n,
                                      float *grad, float *loss, void *stream);

/* Failure-detection check (not part of the paper).  Every wait inside the library's kernels
 * is bounded: the tensor-core kernels poll the mbarrier that tcgen05.commit signals at most
 * a fixed number of times and, when the bound expires, skip the rest of their tile, wait
 * once more (bounded) for the work in flight, release their tensor memory and set an error
 * word that the host reports as POND_ERR_TIMEOUT (pond_sync for the learned predictor, the
 * call itself for training and the stand-alone network calls).  This call exercises that
 * path without a fault: one CTA waits on an mbarrier that nothing arrives on, with `polls`
 * polls (1 .. 2^24) of the same bounded wait, enqueued on `stream` (NULL: the legacy
 * default stream) and waited for.  It returns POND_ERR_TIMEOUT, and the CUDA context stays
 * usable; INVALID_ARG for polls out of range. */
pond_status pond_wait_timeout_check(int64_t polls, void *stream);

/* ---- Kernel-variant autotuning.  Not part of the paper.  Each step kernel is compiled in
   several variants: tile shapes and CTAs per SM of the face corrector, block sizes of the
   cell update, thread counts of the persistent tube kernel.  pond_autotune times every
   variant on this state's own current data (steps timed steps each, after one untimed
   step) and keeps the fastest face and cell (or tube) variant for the following steps;
   on a 1D or 2D grid it then times whole steps of those face and cell kernels against each
   fused step variant and keeps the fastest in `tube` (as pond_set_variants reads it); a
   D3Q64 grid has face tile and cell block variants only (`tube` stays 0).  ms holds
   per-launch times of the face and cell variants and per-step times of the step choices.
   The state is copied aside first (one extra device allocation of the state's size, freed
   before returning) and restored afterwards, so tuning leaves the solution unchanged.
   cache_path (may be NULL) names a text file of "key<TAB>face cell tube" lines; a line
   whose key (device name and SM count, problem kind, precision, size, learned flag)
   matches this state is used without timing, and a new choice is appended.  File errors
   only disable the cache.  Call it outside stream capture.  Errors: INVALID_ARG
   (steps < 1), OOM, CUDA. */
#define POND_TUNE_MAX 32
typedef struct {
    int n;                    /* entries of ms filled (0 when taken from the cache) */
    int face, cell, tube;     /* chosen variant indices */
    int from_cache;           /* 1: the choice came from cache_path */
    double ms[POND_TUNE_MAX]; /* mean ms per launch, in pond_variant_name order */
} pond_tune_result;
pond_status pond_autotune(pond_state *s, int steps, const char *cache_path, pond_tune_result *out);

/* Number of variants of this state and the name of variant i: for a 1D or 2D grid, the
   face variants first, then the cell variants, then the whole-step choices (the separate
   face and cell kernels, then each tile variant of the fused step kernel, which solves a
   tile's faces and updates its cells in one kernel); for a D3Q64 grid, the face tile
   variants, then the cell block variants; for a batch, the tube variants.  The name
   points to a thread-local buffer ("" when i is out of range). */
int pond_variant_count(const pond_state *s);
const char *pond_variant_name(const pond_state *s, int i);

/* Selects variants by index: for a grid face, cell and, in `tube`, the whole step (0: the
   face and cell kernels; k > 0: fused step variant k - 1, used for the plain steps -- the
   learned predictor, pair collection and the equilibration ablation run the face and cell
   kernels); for a D3Q64 grid face and cell (`tube` must be 0); for a batch tube (the others
   are ignored).  Errors: INVALID_ARG for an index out of range. */
pond_status pond_set_variants(pond_state *s, int face, int cell, int tube);

/* Waits for the stream and reports the device diagnostics.  Returns
 * POND_ERR_NONPHYSICAL if any cell or face was non-physical, POND_ERR_NOT_CONVERGED if
 * strict_convergence is set and a face stopped at max_iter, else POND_OK. */
pond_status pond_sync(pond_state *s, pond_diag *diag);

/* Number of kernel launches the library enqueued since pond_init. */
int64_t pond_launch_count(const pond_state *s);

/* Frees everything the state owns (after waiting for its stream). */
void pond_destroy(pond_state *s);

/* Message of the last failed call on this thread. */
const char *pond_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* POND_H */
