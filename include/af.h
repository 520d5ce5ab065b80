/*
 * af.h -- C ABI of the GB300 (sm_103a) implementation of the compact fourth-order,
 * doubly conservative active flux (AF) method with monolithic convex
 * maximum-principle-preserving (MPP) limiting for
 *
 *      u_t + div f(u) = Laplace a(u),   a(u) = int kappa,  kappa >= 0      (Section 1)
 *
 * on periodic Cartesian meshes in 1D, 2D and 3D, on 1D intervals with Dirichlet or
 * outflow ends and on 2D rectangles with outflow ends (arXiv 2510.11527).
 *
 * Degrees of freedom (Section 2 for 1D, Section 4 / Fig. 2 for 2D). All arrays are
 * row-major [ny][nx] with i fastest; a periodic mesh stores nx*ny of each kind:
 *   ub[j][i]  cell average of cell (i,j)
 *   V [j][i]  point value at the corner  (x_{i+1/2}, y_{j+1/2})
 *   X [j][i]  point value at the midpoint of the vertical edge (x_{i+1/2}, y_j)
 *   Y [j][i]  point value at the midpoint of the horizontal edge (x_i, y_{j+1/2})
 * In 1D only ub[i] and P[i] = u(x_{i+1/2}) exist; they are passed in the ub and V
 * slots, and X, Y are ignored (may be NULL). A 1D interval with Dirichlet or outflow
 * ends (grid->bc) has nx+1 point values, P[k] = u(x0 + k dx), k = 0..nx, from the left
 * to the right end; ub keeps nx values. A 2D rectangle with outflow ends has
 * V [ny+1][nx+1] at (x0 + k dx, y0 + l dy), X [ny][nx+1] at (x0 + k dx, y_j) and
 * Y [ny+1][nx] at (x_i, y0 + l dy); ub keeps [ny][nx].
 * 3D (periodic, [nz][ny][nx], i fastest; Section 4): 8 arrays ordered by the kind
 * s = sx + 2 sy + 4 sz of the location (i + sx/2, j + sy/2, k + sz/2): the cell average
 * (s = 0), then the x-face, y-face, xy-edge, z-face, xz-edge, yz-edge and corner values.
 * They are passed through the *_arrays calls below as FP64 (SSP-RK3 / SSP-RK(5,4); zero,
 * linear (p0, p1, p2 velocities) or Burgers flux; blend off or plain). FP32-mixed keeps
 * the averages in FP64 and the 7 point arrays in FP32 on the device (af_device_ptrs_arrays
 * reports the element sizes).
 *
 * Conventions
 *   - Every call returns an af_status. On error the context is left unchanged and
 *     af_last_error() describes the failure; after AF_E_CUDA the context must only be
 *     destroyed.
 *   - Host pointers are read or written synchronously and remain owned by the caller.
 *   - Device work is issued on the stream set by af_set_stream (default: the legacy
 *     default stream). Calls that return host data synchronise that stream.
 *   - There is no CPU fallback: without a usable CUDA device af_create returns
 *     AF_E_UNSUPPORTED.
 */
#ifndef AF_H_
#define AF_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef struct af_ctx af_ctx;   /* opaque; created by af_create, freed by af_destroy */

typedef enum {
  AF_OK = 0,
  AF_E_ARG = -1,          /* invalid argument (sizes, kinds, NULL pointers, bounds)        */
  AF_E_CUDA = -2,         /* a CUDA runtime call failed                                     */
  AF_E_OOM = -3,          /* device allocation failed                                       */
  AF_E_STATE = -4,        /* state outside [umin,umax] beyond the safeguard tolerance, NaN */
  AF_E_CFL = -5,          /* requested dt exceeds the MPP CFL bound of the current state   */
  AF_E_TIMEOUT = -6,      /* a bounded device-side wait gave up                             */
  AF_E_UNSUPPORTED = -7   /* no CUDA device / feature not built                             */
} af_status;

/* Flux kinds (Section 1; examples of Section 6). p[] as listed. */
enum {
  AF_FLUX_ZERO = 0,       /* f = 0                                                          */
  AF_FLUX_LINEAR = 1,     /* f1 = p0 u, f2 = p1 u                                           */
  AF_FLUX_BURGERS = 2,    /* f1 = f2 = p0 u^2                                               */
  AF_FLUX_BL = 3          /* Buckley-Leverett: f1 = u^2/(u^2+(1-u)^2), f2 = f1 (1 - p0 (1-u)^2);
                             in 1D f = f1 (1 - p0 (1-u)^2) (Example 6.6; p0 = 0: no gravity) */
};

/* Diffusion potential kinds a(u) = int kappa (Section 1). */
enum {
  AF_DIFF_NONE = 0,       /* a = 0                                                          */
  AF_DIFF_CONST = 1,      /* a = p0 u                                                       */
  AF_DIFF_PWL = 2,        /* a = p0 min(u - p1, 0) + p2 max(u - p3, 0)  (degenerate band)   */
  AF_DIFF_PME = 3,        /* a = u^p0, p0 integer >= 1 (porous medium)                      */
  AF_DIFF_CUBIC = 4,      /* a = p0 u + p1 u^2 + p2 u^3                                     */
  AF_DIFF_RAMP = 5,       /* a = 0 (u <= p1), p0 (u-p1)^2/(2 p2) (p1 < u < p1+p2),
                             p0 (u - p1 - p2/2) (u >= p1+p2): kappa rises linearly from 0
                             to p0 over [p1, p1+p2], p2 > 0 (Example 6.5: p = 1, 0.5, 0.1) */
  AF_DIFF_CUBIC01 = 6     /* a = p0 v + p1 v^2 + p2 v^3 with v = min(max(u, 0), 1): constant
                             outside [0, 1] (Example 6.6: p = 0, 2 eps, -4 eps / 3)        */
};

/* Ends of a 1D interval (Section 6 uses Dirichlet and outflow ends; their discrete
 * form is this library's reading): ghost cells and ghost points beyond each end.
 * DIRICHLET: every ghost value is the boundary value (bc_left / bc_right) and the two
 * end point values are held at it. OUTFLOW: the DoFs are reflected evenly about the
 * end point (zero gradient); the end point values evolve like interior ones. The CFL
 * maximum includes the two end faces. A 2D rectangle takes OUTFLOW on all four sides
 * (each DoF kind reflected about the side lines) or is periodic. */
enum { AF_BC_PERIODIC = 0, AF_BC_DIRICHLET = 1, AF_BC_OUTFLOW = 2 };

/* Discretisation of the diffusion term. DC: the doubly conservative form (Section
 * 2.2; the default). NODC: the compact form without double conservation of Appendix A
 * (1D, blend off): the cell average receives the face flux kappa(u) D_c(u) at x_{i+1/2},
 * the point value 4/dx^2 sum_{m,n} b_mn kappa(u_m) u_n on its 5-point line; with the
 * limiter on, the total face flux is blended with the low-order face flux
 * F^L - (a(ub_{i+1}) - a(ub_i))/dx by Theta with factor 2. */
enum { AF_FORM_DC = 0, AF_FORM_NODC = 1 };

enum { AF_PREC_FP64 = 0, AF_PREC_FP32_MIXED = 1 };   /* FP32 points/stencils, FP64 averages */
enum { AF_RK_SSP3 = 3, AF_RK_SSP54 = 54 };
enum { AF_BLEND_OFF = 0, AF_BLEND_PLAIN = 1, AF_BLEND_EXTERNAL = 2 };

typedef struct {
  int dim;                /* 1, 2 or 3                                                     */
  int nx, ny;
  double x0, x1, y0, y1;
  int bc;                 /* AF_BC_*: DIRICHLET needs dim = 1; OUTFLOW dim 1 or 2; nx, ny >= 4 */
  double bc_left, bc_right; /* Dirichlet values at x0 and x1                               */
  int nz;                 /* 3D: cells along z                                              */
  double z0, z1;
} af_grid;
typedef struct { int kind; double p[4]; } af_flux;
typedef struct { int kind; double p[4]; } af_diff;
typedef struct { double umin, umax; int from_initial_data; } af_bounds_t;

typedef struct {
  int precision;          /* AF_PREC_FP64 or AF_PREC_FP32_MIXED                             */
  int rk;                 /* AF_RK_SSP3 or AF_RK_SSP54                                      */
  double cfl;             /* C in dt = C / max(alpha/h + kappa_max/h^2); <= 0 -> 0.33/dim    */
  double cfl_diff;        /* diffusive cap dt <= Cd h^2/kappa_max; < 0 -> off; 0 -> default:
                             0.9 x the unlimited scheme's linear diffusive limit               */
  int limiter;            /* 1: monolithic convex limiter + point projection (Section 5)    */
  int blend;              /* AF_BLEND_*: smoothness-indicator blend (Section 5.1.3)         */
  double gamma;           /* blend strength gamma (1 in the paper's examples)               */
  int diffusion_form;     /* AF_FORM_DC or AF_FORM_NODC                                     */
} af_opts;

/* Create a solver for one mesh. Allocates all device buffers (4 state copies for
 * SSP-RK(5,4), 3 for SSP-RK3). bounds->from_initial_data = 1 defers umin/umax to the
 * min/max of the first af_set_state. Returns AF_E_ARG for nx,ny < 1, dim not 1/2,
 * unknown kinds, umin >= umax, non-periodic ends with nx (or, in 2D, ny) < 4;
 * AF_E_UNSUPPORTED for Dirichlet ends or AF_FORM_NODC in 2D, AF_FORM_NODC with a
 * blend, the external indicator with non-periodic ends, and in 3D anything but a
 * periodic mesh (FP64 or FP32-mixed) with the zero, linear or Burgers flux, AF_FORM_DC
 * and the blend off or plain; AF_E_OOM if allocation fails. */
af_status af_create(const af_grid* grid, const af_flux* flux, const af_diff* diff,
                    const af_bounds_t* bounds, const af_opts* opts, af_ctx** out);
af_status af_destroy(af_ctx* ctx);
const char* af_last_error(const af_ctx* ctx);

/* Issue all device work of this context on `stream` (a cudaStream_t, e.g. PyTorch's
 * current stream). NULL selects the legacy default stream. */
af_status af_set_stream(af_ctx* ctx, void* stream);

/* Copy a host state in (doubles, caller-owned, nx*ny values each, row-major; X and Y
 * ignored in 1D; V holds nx+1 values on a bounded 1D interval; a 2D rectangle with
 * ends takes the V, X, Y shapes given at the top of this file). The arrays are copied to the device and checked there; FP32-mixed
 * contexts then round the point values to nearest float. AF_E_STATE if any value is NaN
 * or, with the limiter on, outside [umin, umax]; the current state is then unchanged.
 * Page-locked host memory copies fastest. Returns after the host arrays have been read
 * (the caller may reuse them). */
af_status af_set_state(af_ctx* ctx, const double* ub, const double* V, const double* X, const double* Y);
/* Copy the current state out into caller-owned doubles (FP32 point values widened
 * exactly; the same array lengths as af_set_state). Synchronous with the context's
 * stream. */
af_status af_get_state(af_ctx* ctx, double* ub, double* V, double* X, double* Y);

/* The state as 2^dim arrays (narr must be 1 << dim): 1D ub, P; 2D ub, V, X, Y (as
 * af_set_state); 3D the 8 arrays by kind. Same checks and ownership as af_set_state /
 * af_get_state / af_device_ptrs; these are the only state calls of a 3D context. */
af_status af_set_state_arrays(af_ctx* ctx, int narr, const double* const* arrays);
af_status af_get_state_arrays(af_ctx* ctx, int narr, double* const* arrays);
af_status af_device_ptrs_arrays(af_ctx* ctx, int narr, void** ptrs, int dtype[2]);

/* Borrowed device pointers of the current state (ub, V, X, Y). dtype[0] is 8 (ub is
 * always FP64); dtype[1] is 8 or 4 for the point arrays. Valid until the next call that
 * steps or destroys the context (a bounded 1D interval: nx+1 point values; a 2D
 * rectangle with ends: its padded device layout, (nx+1) x (ny+1) entries per array,
 * entry (I, J) holding the average of cell (I-1, J-1) and the corner / edge values at
 * that cell's top-right; the averages in row and column 0, X in row 0 and Y in column 0
 * are not DoFs). */
af_status af_device_ptrs(af_ctx* ctx, void* ptrs[4], int dtype[2]);

/* Per-cell external smoothness indicator s (nx*ny doubles, host) used when
 * blend == AF_BLEND_EXTERNAL: it replaces the indicator s of Section 5.1.3 in every
 * direction; the limiter and projection still follow. */
af_status af_set_indicator(af_ctx* ctx, const double* s_host);
af_status af_set_indicator_device(af_ctx* ctx, const double* s_dev);

/* One forward-Euler evaluation state <- FE(state, tau) with limiter, projection and
 * blend as configured, and no RK combination (the building block of Section 5). */
af_status af_forward_euler(af_ctx* ctx, double tau);

/* Stage k (0-based) of the configured SSP-RK scheme (Section 3.2); stages must be
 * issued in order 0..af_num_stages()-1 to complete one step. At k = 0 a dt > 0 sets
 * the step (and advances the time); dt <= 0 keeps the step already on the device
 * (from af_dt_device). Later stages ignore dt. */
af_status af_stage(af_ctx* ctx, int k, double dt);
/* Compute the CFL step of the current state on the device into the context's step
 * slot and advance the simulated time by it; no host synchronisation. */
af_status af_dt_device(af_ctx* ctx);
int af_num_stages(const af_ctx* ctx);

/* One full time step. dt > 0: use it as given. dt <= 0: compute the CFL step on the
 * device (eq. multid_av_pp_dt, capped for diffusive linear stability) without a host
 * round trip; if dt_used is non-NULL the stream is synchronised and dt returned. */
af_status af_step(af_ctx* ctx, double dt, double* dt_used);

/* March to time T from the current time with CFL steps, clipping the last step to
 * land on T; *nsteps (if non-NULL) receives the number of steps taken (0 if the time
 * is already T). The device clips each step and counts them; the host issues steps in
 * chunks of 16 and synchronises once per chunk to read the time (steps issued past T
 * have dt = 0 and change nothing). AF_E_STATE if the CFL step is not positive or a
 * value left [umin, umax] beyond the safeguard tolerance. */
af_status af_run(af_ctx* ctx, double T, long long* nsteps);
af_status af_time(af_ctx* ctx, double* t);       /* simulated time (synchronises) */

/* Diagnostics (deterministic reductions in FP64). */
af_status af_mass(af_ctx* ctx, double* mass);                 /* sum(ub) * dx * dy          */
af_status af_bounds(af_ctx* ctx, double* umin, double* umax); /* over all DoFs              */
af_status af_dt_cfl(af_ctx* ctx, double* dt);                 /* CFL step of current state  */
/* Safeguard statistics since creation: values clamped (excess <= tolerance), errors
 * (excess > tolerance), the largest clamped excess, and the mass the clamps of cell
 * averages moved (sum of |clamped - raw| times dx dy: a bound on their effect on the
 * total mass). Any pointer may be NULL. */
af_status af_stats(af_ctx* ctx, long long* clamps, long long* errors, double* max_excess, double* mass_adjust);
/* The cell averages among those clamps (the rest are point values, which the
 * projection bounds anyway). Each changes the total mass; their mass is af_stats'
 * mass_adjust. In the FP32-mixed form such an excess comes from the FP32 rounding of
 * the limited terms, which the FP64 average update adds exactly (less than an FP32 ulp
 * of the bound); the FP64 form has none on the paper's workloads. NULL allowed. */
af_status af_stats_detail(af_ctx* ctx, long long* avg_clamps);

/* ---- batches of independent meshes -------------------------------------------------
 * A batch holds n independent periodic 2D meshes (uneven sizes; per-instance flux and
 * diffusion parameters and bounds) that share the flux kind, precision, RK scheme,
 * limiter, blend and CFL options of *opts (AF_FORM_DC and periodic grids, else
 * AF_E_UNSUPPORTED; blend AF_BLEND_EXTERNAL takes its indicator from a network
 * attached with af_batch_set_mlp). One persistent launch per RK
 * stage walks the (instance, tile) work list with the same tile computation as the
 * single-mesh kernel, so every instance evolves as a single-mesh context with the same
 * options does (bit for bit with SSP-RK3; to a few ulp with SSP-RK(5,4), where the two
 * compilations may contract multiply-adds differently). Per-instance CFL steps and times stay on the device;
 * a full time step is captured once as a CUDA graph and replayed. The batch owns a
 * non-blocking stream unless af_batch_set_stream gives it one. */
typedef struct af_batch af_batch;
af_status af_batch_create(int n, const af_grid* grids, const af_flux* fluxes, const af_diff* diffs,
                          const af_bounds_t* bounds, const af_opts* opts, af_batch** out);
af_status af_batch_destroy(af_batch* b);
const char* af_batch_last_error(const af_batch* b);
af_status af_batch_set_stream(af_batch* b, void* stream);
/* cells in total, work items, current tile shape */
af_status af_batch_info(const af_batch* b, long long* cells, int* tiles, int* tx, int* ty);
/* tile shapes built: 32x8, 64x4, 16x16 */
af_status af_batch_set_tile(af_batch* b, int tx, int ty);
/* time one step with every tile shape on this batch, keep the fastest; the state, the
 * times and the statistics are restored afterwards */
af_status af_batch_autotune(af_batch* b, int* tx, int* ty);
af_status af_batch_set_state(af_batch* b, int i, const double* ub, const double* V, const double* X, const double* Y);
af_status af_batch_get_state(af_batch* b, int i, double* ub, double* V, double* X, double* Y);
af_status af_batch_device_ptrs(af_batch* b, int i, void* ptrs[4], int dtype[2]);
/* nsteps full SSP-RK steps of every instance with its own CFL step (graph replays, no
 * host synchronisation) */
af_status af_batch_step(af_batch* b, int nsteps);
af_status af_batch_sync(af_batch* b);
af_status af_batch_time(af_batch* b, int i, double* t);
af_status af_batch_mass(af_batch* b, int i, double* mass);
af_status af_batch_bounds(af_batch* b, int i, double* umin, double* umax);
af_status af_batch_stats(af_batch* b, long long* clamps, long long* errors, double* max_excess);

/* ---- learned smoothness indicator -------------------------------------------------
 * A 21 -> 32 -> 32 -> 1 network (ReLU hidden layers, softplus output) maps the
 * normalised patch of a cell -- 13 cell averages ub(i+a, j+b), (a,b) in {-1,0,1}^2 and
 * (+-2,0), (0,+-2), then the 8 point values V(i-1,j-1), V(i,j-1), V(i-1,j), V(i,j),
 * X(i-1,j), X(i,j), Y(i,j-1), Y(i,j), each as (v - ub_ij) / (max|v| + 1e-13) -- to s >= 0,
 * which replaces the smoothness indicator s of the blend (Section 5.1.3, direction by
 * direction in 2D). The limiter and projection still follow, so bounds and
 * conservation hold regardless of the network. The two hidden layers run on tensor
 * cores with bf16 inputs/weights and FP32 accumulation; training (forward, backward,
 * Adam) runs in FP32 with the same bf16 rounding points. Parameters are a flat FP32
 * array of AF_MLP_NPARAM values: W1[32][21], b1[32], W2[32][32], b2[32], w3[32], b3.
 * Not in the paper: the paper's indicator is the plain one, which also provides the
 * training labels (max of the two directional indicators). */
#define AF_MLP_NPARAM 1793
typedef struct af_mlp af_mlp;
af_status af_mlp_create(af_mlp** out);
af_status af_mlp_destroy(af_mlp* net);
af_status af_mlp_set_params(af_mlp* net, const float* host, int n);   /* resets Adam state */
af_status af_mlp_get_params(const af_mlp* net, float* host);
/* features (nx*ny x 21, FP32, device) of a 2D context's current state and, if label_dev
 * is non-NULL, the plain indicator's label per cell (device FP32) */
af_status af_mlp_features(af_ctx* ctx, float* feat_dev, float* label_dev);
/* network output for n feature rows (device in, device out) */
af_status af_mlp_infer(const af_mlp* net, const float* feat_dev, long long n, float* out_dev);
/* fused inference (patch gather + network) on a context's current state -> s_dev */
af_status af_mlp_indicator(const af_mlp* net, af_ctx* ctx, double* s_dev);
/* gradient of the mean squared error over the first nsamples rows (no update) */
af_status af_mlp_grad(af_mlp* net, const float* feat_dev, const float* label_dev, int nsamples, float* grad_host,
                      float* loss_host);
/* `steps` Adam steps (lr, betas 0.9/0.999, eps 1e-8) on minibatches of `batch` rows
 * drawn with a counter-based generator (splitmix64) from `seed`; seed 0 takes rows
 * 0..batch-1 in order. Loss of the last batch returned. */
af_status af_mlp_train(af_mlp* net, const float* feat_dev, const float* label_dev, long long nsamples, int batch,
                       int steps, float lr, unsigned long long seed, float* loss_host);
/* attach (or detach with NULL) a network to a 2D context created with
 * blend = AF_BLEND_EXTERNAL: every stage then computes s from its input state first */
af_status af_set_mlp(af_ctx* ctx, const af_mlp* net);
/* the same for a batch created with blend = AF_BLEND_EXTERNAL: before every stage one
 * launch computes s for all instances from their input states (the fused inference of
 * af_mlp_indicator, tile by tile over the batch), then the blended stage reads it. The
 * network is used in place (its later parameter updates take effect at the next stage)
 * and must outlive the batch or be detached first. Waits for the batch's stream.
 * AF_E_STATE for a batch created with another blend; af_batch_step and
 * af_batch_autotune return AF_E_STATE while no network is attached. */
af_status af_batch_set_mlp(af_batch* b, const af_mlp* net);

/* Allocation-free total mass: *mass = cell_area * sum(ub_dev[0..ncells-1]) for a
 * caller-owned device array of cell averages, without any context and without
 * allocating device memory. The paper has no counterpart: this entry point is for
 * callers that cannot call cudaMalloc -- for example a host application whose memory
 * pool has claimed (nearly) all device memory up front, a latency-critical loop that
 * cannot afford the implicit device synchronisation of an allocation, or a plugin host
 * that forbids a library from allocating on its own.
 *   - Scratch: a file-scope device array of AF_MASS_NOALLOC_MAX_CELLS / 2048 partial
 *     sums (512 KiB) plus one result slot, held by every GPU that loads the library
 *     until the process exits. All slots a call uses are overwritten by that call.
 *   - When the array is allocated: with CUDA's default lazy module loading, when its
 *     module is loaded on a device -- at the first call on that device (which resolves
 *     the array's device address, with that device current). A caller whose memory pool
 *     is about to claim the device should therefore make one call first; after that,
 *     calls allocate nothing. The address is resolved again on every call, so the entry
 *     point stays valid after the caller resets the device.
 *   - Calls that overlap on the GPU (e.g. on two streams) race on the shared scratch and
 *     must be serialised by the caller.
 *   - The summation order is fixed (2048-cell blocks, then a fixed tree), so repeated
 *     calls on the same data return bit-identical results; the order differs from
 *     af_mass, so the two agree to FP64 round-off.
 *   - Returns AF_E_ARG for NULL pointers, ncells <= 0 or ncells >
 *     AF_MASS_NOALLOC_MAX_CELLS, or a ub_dev that is not device memory of the current
 *     device (host memory, another GPU's memory); AF_E_CUDA if a launch or copy fails.
 *     Work is issued on `stream` (NULL: legacy default stream), which is synchronised
 *     before returning. */
#define AF_MASS_NOALLOC_MAX_CELLS 134217728LL
af_status af_mass_noalloc(const double* ub_dev, long long ncells, double cell_area, double* mass, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* AF_H_ */
