// Host driver of libaf: contexts, device buffers, SSP-RK stage sequencing, CFL time
// step and diagnostics behind the C ABI of include/af.h (arXiv 2510.11527).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "af.h"
#include "launch.h"
#include "model_host.h"
#include "reduce.cuh"
#include "state_io.cuh"

using af::DevModel;
using af::DevStats;
using af::StageArgs2D;

namespace {


// 0.9 x the linear stability limit kappa dt / h^2 of the unlimited scheme for pure
// diffusion: 1D from the von Neumann analysis of Section 3.2 (0.157 SSP-RK3, 0.333
// SSP-RK(5,4)); 2D from the 4x4 Fourier symbol of the 2D scheme, whose spectral radius
// is 40.78 kappa/h^2 (0.0616 SSP-RK3, 0.1307 SSP-RK(5,4)); 3D from its 8x8 symbol.
// Default diffusive cap: 0.9 x the linear diffusive stability limit of the unlimited
// scheme (with or without the limiter: at the printed C = 0.33/d alone the high-order
// scheme is linearly unstable where kappa dt / h^2 exceeds that limit, which the
// limiter bounds but pays for in accuracy).
double default_cfl_diff(int dim, int rk, int /*limiter*/) {
  if (dim == 1) return 0.9 * (rk == AF_RK_SSP54 ? 0.333 : 0.157);
  // 3D: spectral radius 63.335 kappa/h^2 of the 8x8 symbol; SSP-RK3 / SSP-RK(5,4)
  // stability intervals 2.5127 / 5.330 on the negative real axis
  if (dim == 3) return 0.9 * (rk == AF_RK_SSP54 ? 5.330 : 2.5127) / 63.335;
  return 0.9 * (rk == AF_RK_SSP54 ? 0.1307 : 0.0616);
}

}  // namespace

#include "ctx.h"

#define FAIL(ctx, code, ...)                                  \
  do {                                                        \
    if (ctx) snprintf((ctx)->err, sizeof((ctx)->err), __VA_ARGS__); \
    return code;                                              \
  } while (0)

#define CK(ctx, call)                                                                 \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) FAIL(ctx, AF_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

namespace {

size_t pt_size(const af_ctx* c) { return c->prec == AF_PREC_FP64 ? sizeof(double) : sizeof(float); }

// a 2D rectangle with ends (padded device layout)
bool is_rect(const af_ctx* c) { return c->dim == 2 && c->grid.bc != AF_BC_PERIODIC; }

// values per host array of af_set_state / af_get_state: ub, V, X, Y
void host_sizes(const af_ctx* c, size_t sz[4]) {
  const size_t nx = c->nx, ny = c->ny;
  sz[0] = c->n;
  if (is_rect(c)) {
    sz[1] = (nx + 1) * (ny + 1);
    sz[2] = (nx + 1) * ny;
    sz[3] = nx * (ny + 1);
  } else {
    sz[1] = sz[2] = sz[3] = c->np;
  }
}

template <class PT>
StageArgs2D<PT> base_args(af_ctx* c, int in) {
  StageArgs2D<PT> a;
  std::memset(&a, 0, sizeof(a));
  a.nx = c->pnx;   // the stage kernels tile the padded layout of a 2D rectangle with ends
  a.ny = c->pny;
  a.inv_h1 = c->inv_h1;
  a.inv_h2 = c->inv_h2;
  a.i6h[0] = c->inv_h1 / 6.0;
  a.i6h[1] = c->inv_h2 / 6.0;
  a.i3h2[0] = c->inv_h1 * c->inv_h1 / 3.0;
  a.i3h2[1] = c->inv_h2 * c->inv_h2 / 3.0;
  for (int l = 0; l < 2; ++l) {
    a.i6hf[l] = (float)a.i6h[l];
    a.i3h2f[l] = (float)a.i3h2[l];
  }
  a.ub = c->ub[in];
  a.V = (const PT*)c->pv[in];
  a.X = (const PT*)c->px[in];
  a.Y = (const PT*)c->py[in];
  a.dt = c->dt_dev;
  a.s_ext = (c->s_ext_user && !c->mlp) ? c->s_ext_user : c->s_ext;
  // the plain indicator of the column-marching FP32 stage: s_1, s_2 as FP32 in the
  // indicator scratch (n doubles), which the plain blend does not use otherwise
  a.sb[0] = (const float*)c->s_ext;
  a.sb[1] = (const float*)c->s_ext + c->n;
  a.limiter = c->opts.limiter;
  a.blend = c->opts.blend;
  a.blend_external = c->opts.blend == AF_BLEND_EXTERNAL;
  a.gamma = c->opts.gamma;
  a.tol = c->tol;
  a.stats = c->stats;
  a.bc = c->grid.bc;
  a.bc_left = c->grid.bc_left;
  a.bc_right = c->grid.bc_right;
  a.nodc = c->opts.diffusion_form == AF_FORM_NODC;
  return a;
}

// output k of a stage: out = cA * U[aidx] + cF * FE(in, tcoef * dt) -> U[oidx]
template <class PT>
void set_out(af_ctx* c, StageArgs2D<PT>& a, int k, int oidx, double cA, int aidx, double cF, double tcoef, int sg) {
  a.tcoef[k] = tcoef;
  a.cA[k] = cA;
  a.cF[k] = cF;
  a.Aub[k] = aidx >= 0 ? c->ub[aidx] : nullptr;
  a.AV[k] = aidx >= 0 ? (const PT*)c->pv[aidx] : nullptr;
  a.AX[k] = aidx >= 0 ? (const PT*)c->px[aidx] : nullptr;
  a.AY[k] = aidx >= 0 ? (const PT*)c->py[aidx] : nullptr;
  a.Oub[k] = c->ub[oidx];
  a.OV[k] = (PT*)c->pv[oidx];
  a.OX[k] = (PT*)c->px[oidx];
  a.OY[k] = (PT*)c->py[oidx];
  a.sg[k] = sg;
  a.nout = k + 1;
}

// With a learned indicator attached, the network first computes s from the stage's
// input state into the context's indicator array, which the stage kernel then reads.
template <class PT>
cudaError_t run_indicator(af_ctx* c, const StageArgs2D<PT>& a) {
  if (!c->mlp) return cudaSuccess;
  int in = 0;
  while (in < c->nbuf && c->ub[in] != a.ub) ++in;
  return af::mlp_indicator_launch(c, c->mlp, in, c->s_ext);
}

template <class PT>
cudaError_t launch(af_ctx* c, const StageArgs2D<PT>& a);
template <>
cudaError_t launch<double>(af_ctx* c, const StageArgs2D<double>& a) {
  cudaError_t e = run_indicator(c, a);
  if (e != cudaSuccess) return e;
  if (c->dim == 1) return af::launch_stage1d_f64(c->flux.kind, c->m, a, c->stream);
  if (is_rect(c)) return af::launch_stage2d_rect_f64(c->flux.kind, c->opts.blend != AF_BLEND_OFF, c->m, a, c->stream);
  return af::launch_stage2d_f64(c->flux.kind, c->opts.blend != AF_BLEND_OFF, c->m, a, c->stream);
}
template <>
cudaError_t launch<float>(af_ctx* c, const StageArgs2D<float>& a) {
  cudaError_t e = run_indicator(c, a);
  if (e != cudaSuccess) return e;
  if (c->dim == 1) return af::launch_stage1d_f32(c->flux.kind, c->m, a, c->stream);
  if (is_rect(c)) return af::launch_stage2d_rect_f32(c->flux.kind, c->opts.blend != AF_BLEND_OFF, c->m, a, c->stream);
  return af::launch_stage2d_f32(c->flux.kind, c->opts.blend != AF_BLEND_OFF, c->m, a, c->stream);
}

// Buffer roles of stage k of the configured scheme (see af_stage): the input buffer and
// one or two outputs out = cA * U[aidx] + cF * FE(U[in], tcoef * dt) -> U[oidx]; sg:
// apply the post-stage safeguard. Returns the number of outputs (0: k out of range).
struct OutSpec {
  int oidx;
  double cA;
  int aidx;
  double cF, tcoef;
  int sg;
};
int stage_plan(const af_ctx* c, int k, int* in, OutSpec out[2]) {
  if (c->opts.rk == AF_RK_SSP3) {
    if (k == 0) { *in = 0; out[0] = {1, 0.0, -1, 1.0, 1.0, 1}; return 1; }
    if (k == 1) { *in = 1; out[0] = {2, 0.75, 0, 0.25, 1.0, 1}; return 1; }
    if (k == 2) { *in = 2; out[0] = {0, 1.0 / 3.0, 0, 2.0 / 3.0, 1.0, 1}; return 1; }
    return 0;
  }
  const double(*A)[5] = af::kA54;
  const double(*B)[5] = af::kB54;
  switch (k) {
    case 0: *in = 0; out[0] = {1, 0.0, -1, A[0][0], B[0][0] / A[0][0], 1}; return 1;
    case 1: *in = 1; out[0] = {2, A[1][0], 0, A[1][1], B[1][1] / A[1][1], 1}; return 1;
    case 2: *in = 2; out[0] = {3, A[2][0], 0, A[2][2], B[2][2] / A[2][2], 1}; return 1;
    case 3:
      // u^(4) = a30 u0 + a33 FE(u3); partial = a42 u2 + a43 FE(u3, own ratio) in place
      *in = 3;
      out[0] = {1, A[3][0], 0, A[3][3], B[3][3] / A[3][3], 1};
      out[1] = {2, A[4][2], 2, A[4][3], B[4][3] / A[4][3], 0};
      return 2;
    case 4: *in = 1; out[0] = {0, 1.0, 2, A[4][4], B[4][4] / A[4][4], 1}; return 1;
    default: return 0;
  }
}

// stage k of the configured scheme
template <class PT>
af_status stage_impl(af_ctx* c, int k) {
  int in = 0;
  OutSpec out[2];
  const int nout = stage_plan(c, k, &in, out);
  if (nout == 0) FAIL(c, AF_E_ARG, "stage %d out of range", k);
  auto a = base_args<PT>(c, in);
  for (int o = 0; o < nout; ++o) set_out<PT>(c, a, o, out[o].oidx, out[o].cA, out[o].aidx, out[o].cF, out[o].tcoef, out[o].sg);
  CK(c, launch<PT>(c, a));
  return AF_OK;
}

// the 3D stage arguments for input buffer `in` (outputs added by the caller); T is the
// context's point / stencil precision
template <class T>
af::StageArgs3D<T> args3d(af_ctx* c, int in) {
  af::StageArgs3D<T> a;
  std::memset(&a, 0, sizeof(a));
  a.n[0] = c->nx;
  a.n[1] = c->ny;
  a.n[2] = c->nz;
  a.inv_h[0] = c->inv_h1;
  a.inv_h[1] = c->inv_h2;
  a.inv_h[2] = c->inv_h3;
  for (int l = 0; l < 3; ++l) {
    a.i6h[l] = a.inv_h[l] / 6.0;
    a.i3h2[l] = a.inv_h[l] * a.inv_h[l] / 3.0;
    a.inv_hT[l] = (T)a.inv_h[l];
    a.i6hT[l] = (T)a.i6h[l];
    a.i3h2T[l] = (T)a.i3h2[l];
  }
  a.ub = (const double*)c->k3[in][0];
  for (int s = 1; s < 8; ++s) a.pt[s] = (const T*)c->k3[in][s];
  a.dt = c->dt_dev;
  a.limiter = c->opts.limiter;
  a.blend = c->opts.blend;
  a.gamma = c->opts.gamma;
  a.tol = c->tol;
  a.stats = c->stats;
  a.C = (T*)c->scr3[0];
  for (int l = 0; l < 3; ++l) {
    a.FH[l] = (T*)c->scr3[1 + l];
    a.AH[l] = (T*)c->scr3[4 + l];
    a.FL[l] = (T*)c->scr3[7 + l];
    a.S[l] = (T*)c->scr3[10 + l];
    a.Flim[l] = (T*)c->scr3[13 + l];
    a.Alim[l] = (T*)c->scr3[16 + l];
  }
  return a;
}

template <class T>
af_status stage3d_typed(af_ctx* c, int in, const OutSpec* out, int nout) {
  af::StageArgs3D<T> a = args3d<T>(c, in);
  a.nout = nout;
  for (int o = 0; o < nout; ++o) {
    a.tcoef[o] = out[o].tcoef;
    a.cA[o] = out[o].cA;
    a.cF[o] = out[o].cF;
    a.sg[o] = out[o].sg;
    a.Aub[o] = out[o].aidx >= 0 ? (const double*)c->k3[out[o].aidx][0] : nullptr;
    a.Oub[o] = (double*)c->k3[out[o].oidx][0];
    for (int s = 1; s < 8; ++s) {
      a.Apt[o][s] = out[o].aidx >= 0 ? (const T*)c->k3[out[o].aidx][s] : nullptr;
      a.Opt[o][s] = (T*)c->k3[out[o].oidx][s];
    }
  }
  if constexpr (sizeof(T) == 8) {
    CK(c, af::launch_stage3d_f64(c->flux.kind, c->m, a, c->stream));
  } else {
    CK(c, af::launch_stage3d_f32(c->flux.kind, c->m, a, c->stream));
  }
  return AF_OK;
}

af_status stage3d_out(af_ctx* c, int in, const OutSpec* out, int nout) {
  return c->prec == AF_PREC_FP64 ? stage3d_typed<double>(c, in, out, nout) : stage3d_typed<float>(c, in, out, nout);
}

af_status stage3d_impl(af_ctx* c, int k) {
  int in = 0;
  OutSpec out[2];
  const int nout = stage_plan(c, k, &in, out);
  if (nout == 0) FAIL(c, AF_E_ARG, "stage %d out of range", k);
  return stage3d_out(c, in, out, nout);
}

af_status stage_any(af_ctx* c, int k) {
  if (c->dim == 3) return stage3d_impl(c, k);
  return c->prec == AF_PREC_FP64 ? stage_impl<double>(c, k) : stage_impl<float>(c, k);
}

template <int FLUX>
cudaError_t launch_rate(af_ctx* c) {
  const int blocks = 152 * 4;
  if constexpr (FLUX == af::FLUX_BL)
    af::dt_rate_kernel<FLUX><<<blocks, af::RED_THREADS, 0, c->stream>>>(c->m, c->dim, c->pnx, c->pny, c->inv_h1,
                                                                         c->inv_h2, c->kmax, c->ub[0], c->rate_bits,
                                                                         c->grid.bc, c->grid.bc_left, c->grid.bc_right);
  else
    af::dt_rate_maxu_kernel<FLUX><<<blocks, af::RED_THREADS, 0, c->stream>>>(
        c->m, c->dim, c->pnx, c->pny, c->inv_h1, c->inv_h2, c->kmax, c->ub[0], c->rate_bits, c->grid.bc,
        c->grid.bc_left, c->grid.bc_right);
  return cudaGetLastError();
}

// device CFL step -> *dst (no host round trip); t_acc: advance the device time
af_status dt_device(af_ctx* c, double* dst, double* t_acc, double t_end = -1.0, double* count = nullptr) {
  cudaError_t e;
  if (c->dim == 3) {
    const int n3[3] = {c->nx, c->ny, c->nz};
    const double ih3[3] = {c->inv_h1, c->inv_h2, c->inv_h3};
    CK(c, af::launch_rate3d(c->flux.kind, c->m, n3, (const double*)c->k3[0][0], ih3, c->kmax, c->rate_bits, c->stream));
    const double hmin = std::min(c->dx, std::min(c->dy, c->dz));
    // no interior extrema of f_l' in 3D: the finalize step adds no extremum terms (dim 0)
    af::dt_finalize_kernel<<<1, 1, 0, c->stream>>>(c->rate_bits, c->m, 0, c->inv_h1, c->inv_h2, c->cfl, c->cfl_diff,
                                                   c->kmax, 1.0 / (hmin * hmin), dst, t_acc, t_end, count);
    CK(c, cudaGetLastError());
    return AF_OK;
  }
  switch (c->flux.kind) {
    case AF_FLUX_ZERO: e = launch_rate<af::FLUX_ZERO>(c); break;
    case AF_FLUX_LINEAR: e = launch_rate<af::FLUX_LINEAR>(c); break;
    case AF_FLUX_BURGERS: e = launch_rate<af::FLUX_BURGERS>(c); break;
    default: e = launch_rate<af::FLUX_BL>(c); break;
  }
  CK(c, e);
  const double hmin = c->dim == 1 ? c->dx : std::min(c->dx, c->dy);
  af::dt_finalize_kernel<<<1, 1, 0, c->stream>>>(c->rate_bits, c->m, c->dim, c->inv_h1, c->inv_h2, c->cfl,
                                                 c->cfl_diff, c->kmax, 1.0 / (hmin * hmin), dst, t_acc, t_end, count);
  CK(c, cudaGetLastError());
  return AF_OK;
}

af_status read_scalar(af_ctx* c, const double* dev, double* out) {
  CK(c, cudaMemcpyAsync(c->host_pinned, dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  *out = c->host_pinned[0];
  return AF_OK;
}

// reduction of x[0, count) (op 0 sum, 1 min, 2 max); with w > 0 only the entries whose
// column (of rows of width w) is >= ilo and row >= jlo
template <class S>
af_status reduce_array(af_ctx* c, const S* x, size_t count, int op, double init, double* out_dev, int accumulate,
                       int w = 0, int ilo = 0, int jlo = 0) {
  const int blocks = (int)std::min<size_t>(af::RED_MAX_BLOCKS, (count + af::RED_THREADS - 1) / af::RED_THREADS);
  if (w > 0)
    af::partial_masked_kernel<S><<<blocks, af::RED_THREADS, 0, c->stream>>>(x, count, w, ilo, jlo, op, init,
                                                                            c->partial);
  else
    af::partial_kernel<S><<<blocks, af::RED_THREADS, 0, c->stream>>>(x, count, op, init, c->partial);
  CK(c, cudaGetLastError());
  af::finalize_kernel<<<1, af::RED_THREADS, 0, c->stream>>>(c->partial, blocks, op, out_dev, accumulate);
  CK(c, cudaGetLastError());
  return AF_OK;
}

af_status set_dt(af_ctx* c, double dt, bool advance) {
  af::set_dt_kernel<<<1, 1, 0, c->stream>>>(c->dt_dev, advance ? c->t_dev : nullptr, dt);
  CK(c, cudaGetLastError());
  return AF_OK;
}

}  // namespace

extern "C" {

af_status af_create(const af_grid* grid, const af_flux* flux, const af_diff* diff, const af_bounds_t* bounds,
                    const af_opts* opts, af_ctx** out) {
  if (!grid || !flux || !diff || !bounds || !opts || !out) return AF_E_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return AF_E_UNSUPPORTED;
  if (grid->dim < 1 || grid->dim > 3) return AF_E_ARG;
  if (grid->nx < 1 || (grid->dim >= 2 && grid->ny < 1) || (grid->dim == 3 && grid->nz < 1)) return AF_E_ARG;
  if (!(grid->x1 > grid->x0) || (grid->dim >= 2 && !(grid->y1 > grid->y0)) ||
      (grid->dim == 3 && !(grid->z1 > grid->z0)))
    return AF_E_ARG;
  if (flux->kind < AF_FLUX_ZERO || flux->kind > AF_FLUX_BL) return AF_E_ARG;
  if (diff->kind < AF_DIFF_NONE || diff->kind > AF_DIFF_CUBIC01) return AF_E_ARG;
  if (diff->kind == AF_DIFF_PME && (diff->p[0] < 1.0 || diff->p[0] != std::floor(diff->p[0]))) return AF_E_ARG;
  if (diff->kind == AF_DIFF_RAMP && !(diff->p[2] > 0.0)) return AF_E_ARG;
  if (grid->bc < AF_BC_PERIODIC || grid->bc > AF_BC_OUTFLOW) return AF_E_ARG;
  if (opts->diffusion_form != AF_FORM_DC && opts->diffusion_form != AF_FORM_NODC) return AF_E_ARG;
  if (grid->bc == AF_BC_DIRICHLET && grid->dim != 1) return AF_E_UNSUPPORTED;
  if (grid->bc != AF_BC_PERIODIC && (grid->nx < 4 || (grid->dim == 2 && grid->ny < 4))) return AF_E_ARG;
  if (opts->diffusion_form == AF_FORM_NODC && (grid->dim != 1 || opts->blend != AF_BLEND_OFF)) return AF_E_UNSUPPORTED;
  if (grid->bc != AF_BC_PERIODIC && opts->blend == AF_BLEND_EXTERNAL) return AF_E_UNSUPPORTED;
  if (grid->dim == 3 && (double)grid->nx * grid->ny * grid->nz >= 2147483648.0) return AF_E_ARG;   // 32-bit cell index
  if (grid->dim == 3 && (grid->bc != AF_BC_PERIODIC || flux->kind == AF_FLUX_BL ||
                         opts->blend == AF_BLEND_EXTERNAL || opts->diffusion_form != AF_FORM_DC))
    return AF_E_UNSUPPORTED;
  if (!bounds->from_initial_data && !(bounds->umax > bounds->umin)) return AF_E_ARG;
  if (opts->precision != AF_PREC_FP64 && opts->precision != AF_PREC_FP32_MIXED) return AF_E_ARG;
  if (opts->rk != AF_RK_SSP3 && opts->rk != AF_RK_SSP54) return AF_E_ARG;
  if (opts->blend < AF_BLEND_OFF || opts->blend > AF_BLEND_EXTERNAL) return AF_E_ARG;

  af_ctx* c = new (std::nothrow) af_ctx;
  if (!c) return AF_E_OOM;
  c->grid = *grid;
  c->flux = *flux;
  c->diff = *diff;
  c->bnd = *bounds;
  c->opts = *opts;
  c->dim = grid->dim;
  c->nx = grid->nx;
  c->ny = grid->dim >= 2 ? grid->ny : 1;
  c->nz = grid->dim == 3 ? grid->nz : 1;
  c->n = (size_t)c->nx * c->ny * c->nz;
  c->np = c->n + (grid->dim == 1 && grid->bc != AF_BC_PERIODIC ? 1 : 0);
  const bool rect = grid->dim == 2 && grid->bc != AF_BC_PERIODIC;
  c->pnx = c->nx + (rect ? 1 : 0);
  c->pny = c->ny + (rect ? 1 : 0);
  c->pn = (size_t)c->pnx * c->pny;
  c->prec = opts->precision;
  c->nbuf = opts->rk == AF_RK_SSP54 ? 4 : 3;
  c->dx = (grid->x1 - grid->x0) / grid->nx;
  c->dy = grid->dim >= 2 ? (grid->y1 - grid->y0) / grid->ny : 1.0;
  c->dz = grid->dim == 3 ? (grid->z1 - grid->z0) / grid->nz : 1.0;
  c->inv_h1 = 1.0 / c->dx;
  c->inv_h2 = grid->dim >= 2 ? 1.0 / c->dy : 0.0;
  c->inv_h3 = grid->dim == 3 ? 1.0 / c->dz : 0.0;
  c->cfl = opts->cfl > 0.0 ? opts->cfl : 0.33 / grid->dim;
  c->cfl_diff = opts->cfl_diff > 0.0 ? opts->cfl_diff : (opts->cfl_diff < 0.0 ? 0.0 : default_cfl_diff(c->dim, opts->rk, opts->limiter));
  std::memset(&c->m, 0, sizeof(c->m));
  c->m.flux_kind = flux->kind;
  c->m.diff_kind = diff->kind;
  for (int k = 0; k < 4; ++k) { c->m.fp[k] = flux->p[k]; c->m.dp[k] = diff->p[k]; }
  c->bounds_pending = bounds->from_initial_data != 0;
  c->m.umin = bounds->umin;
  c->m.umax = bounds->umax;
  af::finish_model(c->m, flux->kind, grid->dim);
  if (!c->bounds_pending) c->kmax = af::kappa_max_of(*diff, bounds->umin, bounds->umax);
  const double scale = std::max(std::fabs(bounds->umin), std::fabs(bounds->umax));
  c->tol = (c->prec == AF_PREC_FP64 ? 8.0 * 2.220446049250313e-16 : 64.0 * 1.1920929e-07) * scale;

  // one device allocation: nbuf states + scratch
  const size_t ps = pt_size(c);
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t ulen = rect ? c->pn : c->n, plen = rect ? c->pn : c->np;
  const bool d3 = grid->dim == 3;
  // 3D: the FP64 averages and 7 point arrays per state, and 19 scratch arrays of the 3D
  // stage (sized for FP64)
  const size_t per_state = d3 ? al(c->n * 8) + 7 * al(c->n * ps) : al(ulen * 8) + 3 * al(plen * ps);
  const size_t scr3 = d3 ? 19 * al(c->n * 8) : 0;
  const size_t scratch = al(8) * 2 + al(8 * 8) + al(8 * af::RED_MAX_BLOCKS) + al(8) + al(sizeof(DevStats)) + al(c->n * 8);
  const size_t total = per_state * c->nbuf + scratch + scr3;
  if (cudaMalloc(&c->block, total) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return AF_E_OOM;
  }
  unsigned char* p = c->block;
  for (int b = 0; b < c->nbuf; ++b) {
    if (d3) {
      for (int s = 0; s < 8; ++s) { c->k3[b][s] = p; p += al(c->n * (s == 0 ? 8 : ps)); }
      c->ub[b] = (double*)c->k3[b][0];
      c->pv[b] = c->k3[b][1];
      c->px[b] = c->k3[b][2];
      c->py[b] = c->k3[b][3];
      continue;
    }
    c->ub[b] = (double*)p; p += al(ulen * 8);
    c->pv[b] = p; p += al(plen * ps);
    c->px[b] = p; p += al(plen * ps);
    c->py[b] = p; p += al(plen * ps);
  }
  c->dt_dev = (double*)p; p += al(8);
  c->t_dev = (double*)p; p += al(8);
  c->red = (double*)p; p += al(8 * 8);
  c->partial = (double*)p; p += al(8 * af::RED_MAX_BLOCKS);
  c->rate_bits = (unsigned long long*)p; p += al(16);
  c->stats = (DevStats*)p; p += al(sizeof(DevStats));
  c->s_ext = (double*)p; p += al(c->n * 8);
  for (int k = 0; d3 && k < 19; ++k) { c->scr3[k] = p; p += al(c->n * 8); }
  if (cudaMemset(c->block, 0, total) != cudaSuccess || cudaMallocHost(&c->host_pinned, 8 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->block);
    delete c;
    return AF_E_OOM;
  }
  *out = c;
  return AF_OK;
}

af_status af_destroy(af_ctx* c) {
  if (!c) return AF_E_ARG;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  cudaFree(c->block);
  cudaFreeHost(c->host_pinned);
  delete c;
  return AF_OK;
}

const char* af_last_error(const af_ctx* c) { return c ? c->err : "null context"; }

af_status af_set_stream(af_ctx* c, void* stream) {
  if (!c) return AF_E_ARG;
  c->stream = (cudaStream_t)stream;
  return AF_OK;
}

int af_num_stages(const af_ctx* c) { return !c ? 0 : (c->opts.rk == AF_RK_SSP54 ? 5 : 3); }

af_status af_set_state(af_ctx* c, const double* ub, const double* V, const double* X, const double* Y) {
  if (!c || !ub || !V || (c->dim == 2 && (!X || !Y))) return AF_E_ARG;
  if (c->dim == 3) FAIL(c, AF_E_ARG, "a 3D state has 8 arrays: use af_set_state_arrays");
  const int na = c->dim == 2 ? 4 : 2;
  const double* src[4] = {ub, V, X, Y};
  size_t sz[4], off[5] = {0, 0, 0, 0, 0};
  host_sizes(c, sz);
  for (int a = 0; a < na; ++a) off[a + 1] = off[a] + sz[a];
  const size_t total = off[na];
  // staging: the RK temporaries (buffers 1..nbuf-1, contiguous, >= 8 total bytes), the
  // host arrays back to back
  double* stg = c->ub[1];
  for (int a = 0; a < na; ++a)
    CK(c, cudaMemcpyAsync(stg + off[a], src[a], sz[a] * 8, cudaMemcpyHostToDevice, c->stream));
  const int nb = (int)std::min<size_t>(af::STATE_IO_BLOCKS, (total + af::RED_THREADS - 1) / af::RED_THREADS);
  af::validate_partial_kernel<<<nb, af::RED_THREADS, 0, c->stream>>>(stg, total, (unsigned long long*)c->partial);
  CK(c, cudaGetLastError());
  af::validate_final_kernel<<<1, af::RED_THREADS, 0, c->stream>>>((const unsigned long long*)c->partial, nb, c->red + 5);
  CK(c, cudaGetLastError());
  CK(c, cudaMemcpyAsync(c->host_pinned, c->red + 5, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  const double nan = c->host_pinned[0], lo = c->host_pinned[1], hi = c->host_pinned[2];
  if (nan > 0.0) FAIL(c, AF_E_STATE, "NaN in the input arrays (%.0f values)", nan);
  if (c->bounds_pending) {
    if (!(hi > lo)) FAIL(c, AF_E_STATE, "bounds from initial data need max > min");
    c->m.umin = lo;
    c->m.umax = hi;
    c->m.umid = 0.5 * (lo + hi);
    c->kmax = af::kappa_max_of(c->diff, lo, hi);
    const double scale = std::max(std::fabs(lo), std::fabs(hi));
    c->tol = (c->prec == AF_PREC_FP64 ? 8.0 * 2.220446049250313e-16 : 64.0 * 1.1920929e-07) * scale;
    c->bounds_pending = false;
  } else if (c->opts.limiter && (lo < c->m.umin || hi > c->m.umax)) {
    FAIL(c, AF_E_STATE, "input outside [umin, umax]: [%g, %g]", lo, hi);
  }
  if (is_rect(c)) {
    const int grid = (int)std::min<size_t>(152 * 8, (c->pn + af::RED_THREADS - 1) / af::RED_THREADS);
    if (c->prec == AF_PREC_FP64)
      af::scatter_rect_kernel<double><<<grid, af::RED_THREADS, 0, c->stream>>>(
          stg, c->nx, c->ny, c->ub[0], (double*)c->pv[0], (double*)c->px[0], (double*)c->py[0]);
    else
      af::scatter_rect_kernel<float><<<grid, af::RED_THREADS, 0, c->stream>>>(
          stg, c->nx, c->ny, c->ub[0], (float*)c->pv[0], (float*)c->px[0], (float*)c->py[0]);
  } else {
    const size_t n = c->n, np = c->np;
    const int grid = (int)std::min<size_t>(152 * 8, (np + af::RED_THREADS - 1) / af::RED_THREADS);
    if (c->prec == AF_PREC_FP64)
      af::scatter_state_kernel<double><<<grid, af::RED_THREADS, 0, c->stream>>>(
          stg, n, np, na, c->ub[0], (double*)c->pv[0], (double*)c->px[0], (double*)c->py[0]);
    else
      af::scatter_state_kernel<float><<<grid, af::RED_THREADS, 0, c->stream>>>(
          stg, n, np, na, c->ub[0], (float*)c->pv[0], (float*)c->px[0], (float*)c->py[0]);
  }
  CK(c, cudaGetLastError());
  return AF_OK;
}

af_status af_get_state(af_ctx* c, double* ub, double* V, double* X, double* Y) {
  if (!c || !ub || !V || (c->dim == 2 && (!X || !Y))) return AF_E_ARG;
  if (c->dim == 3) FAIL(c, AF_E_ARG, "a 3D state has 8 arrays: use af_get_state_arrays");
  const int na = c->dim == 2 ? 4 : 2;
  double* dst[4] = {ub, V, X, Y};
  if (is_rect(c)) {
    // padded device layout -> the caller's layout, as doubles in the staging area
    size_t sz[4], off[5] = {0, 0, 0, 0, 0};
    host_sizes(c, sz);
    for (int a = 0; a < na; ++a) off[a + 1] = off[a] + sz[a];
    double* stg = c->ub[1];
    const int grid = (int)std::min<size_t>(152 * 8, (c->pn + af::RED_THREADS - 1) / af::RED_THREADS);
    if (c->prec == AF_PREC_FP64)
      af::gather_rect_kernel<double><<<grid, af::RED_THREADS, 0, c->stream>>>(
          c->ub[0], (const double*)c->pv[0], (const double*)c->px[0], (const double*)c->py[0], c->nx, c->ny, stg);
    else
      af::gather_rect_kernel<float><<<grid, af::RED_THREADS, 0, c->stream>>>(
          c->ub[0], (const float*)c->pv[0], (const float*)c->px[0], (const float*)c->py[0], c->nx, c->ny, stg);
    CK(c, cudaGetLastError());
    for (int a = 0; a < na; ++a)
      CK(c, cudaMemcpyAsync(dst[a], stg + off[a], sz[a] * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return AF_OK;
  }
  const size_t n = c->n, np = c->np;
  CK(c, cudaMemcpyAsync(ub, c->ub[0], n * 8, cudaMemcpyDeviceToHost, c->stream));
  if (c->prec == AF_PREC_FP64) {
    void* src[3] = {c->pv[0], c->px[0], c->py[0]};
    for (int a = 1; a < na; ++a) CK(c, cudaMemcpyAsync(dst[a], src[a - 1], np * 8, cudaMemcpyDeviceToHost, c->stream));
  } else {
    // FP32 points widened on the device into the staging area, then copied
    double* stg = c->ub[1];
    const int grid = (int)std::min<size_t>(152 * 8, (np + af::RED_THREADS - 1) / af::RED_THREADS);
    af::gather_points_kernel<<<grid, af::RED_THREADS, 0, c->stream>>>(
        (const float*)c->pv[0], (const float*)c->px[0], (const float*)c->py[0], np, na, stg);
    CK(c, cudaGetLastError());
    for (int a = 1; a < na; ++a)
      CK(c, cudaMemcpyAsync(dst[a], stg + (a - 1) * np, np * 8, cudaMemcpyDeviceToHost, c->stream));
  }
  CK(c, cudaStreamSynchronize(c->stream));
  return AF_OK;
}

af_status af_set_state_arrays(af_ctx* c, int narr, const double* const* arrays) {
  if (!c || !arrays || narr != (1 << c->dim)) return AF_E_ARG;
  for (int a = 0; a < narr; ++a)
    if (!arrays[a]) return AF_E_ARG;
  if (c->dim == 1) return af_set_state(c, arrays[0], arrays[1], nullptr, nullptr);
  if (c->dim == 2) return af_set_state(c, arrays[0], arrays[1], arrays[2], arrays[3]);
  // 3D: stage the 8 arrays in the RK temporaries (buffers 1.., contiguous, >= 64 n
  // bytes), check them there, then copy (FP32-mixed: round the points to nearest)
  const size_t n = c->n;
  double* stg = (double*)c->k3[1][0];
  for (int a = 0; a < 8; ++a)
    CK(c, cudaMemcpyAsync(stg + a * n, arrays[a], n * 8, cudaMemcpyHostToDevice, c->stream));
  const size_t total = 8 * n;
  const int nb = (int)std::min<size_t>(af::STATE_IO_BLOCKS, (total + af::RED_THREADS - 1) / af::RED_THREADS);
  af::validate_partial_kernel<<<nb, af::RED_THREADS, 0, c->stream>>>(stg, total, (unsigned long long*)c->partial);
  CK(c, cudaGetLastError());
  af::validate_final_kernel<<<1, af::RED_THREADS, 0, c->stream>>>((const unsigned long long*)c->partial, nb, c->red + 5);
  CK(c, cudaGetLastError());
  CK(c, cudaMemcpyAsync(c->host_pinned, c->red + 5, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  const double nan = c->host_pinned[0], lo = c->host_pinned[1], hi = c->host_pinned[2];
  if (nan > 0.0) FAIL(c, AF_E_STATE, "NaN in the input arrays (%.0f values)", nan);
  if (c->bounds_pending) {
    if (!(hi > lo)) FAIL(c, AF_E_STATE, "bounds from initial data need max > min");
    c->m.umin = lo;
    c->m.umax = hi;
    c->m.umid = 0.5 * (lo + hi);
    c->kmax = af::kappa_max_of(c->diff, lo, hi);
    c->tol = (c->prec == AF_PREC_FP64 ? 8.0 * 2.220446049250313e-16 : 64.0 * 1.1920929e-07) *
             std::max(std::fabs(lo), std::fabs(hi));
    c->bounds_pending = false;
  } else if (c->opts.limiter && (lo < c->m.umin || hi > c->m.umax)) {
    FAIL(c, AF_E_STATE, "input outside [umin, umax]: [%g, %g]", lo, hi);
  }
  CK(c, cudaMemcpyAsync(c->k3[0][0], stg, n * 8, cudaMemcpyDeviceToDevice, c->stream));
  const int grid = (int)std::min<size_t>(152 * 8, (n + af::RED_THREADS - 1) / af::RED_THREADS);
  for (int a = 1; a < 8; ++a) {
    if (c->prec == AF_PREC_FP64) {
      CK(c, cudaMemcpyAsync(c->k3[0][a], stg + a * n, n * 8, cudaMemcpyDeviceToDevice, c->stream));
    } else {
      af::narrow_kernel<<<grid, af::RED_THREADS, 0, c->stream>>>(stg + a * n, (float*)c->k3[0][a], n);
      CK(c, cudaGetLastError());
    }
  }
  return AF_OK;
}

af_status af_get_state_arrays(af_ctx* c, int narr, double* const* arrays) {
  if (!c || !arrays || narr != (1 << c->dim)) return AF_E_ARG;
  for (int a = 0; a < narr; ++a)
    if (!arrays[a]) return AF_E_ARG;
  if (c->dim == 1) return af_get_state(c, arrays[0], arrays[1], nullptr, nullptr);
  if (c->dim == 2) return af_get_state(c, arrays[0], arrays[1], arrays[2], arrays[3]);
  const size_t n = c->n;
  if (c->prec == AF_PREC_FP64) {
    for (int a = 0; a < 8; ++a)
      CK(c, cudaMemcpyAsync(arrays[a], c->k3[0][a], n * 8, cudaMemcpyDeviceToHost, c->stream));
  } else {
    // FP32 points widened on the device into the staging area, then copied
    double* stg = (double*)c->k3[1][0];
    const int grid = (int)std::min<size_t>(152 * 8, (n + af::RED_THREADS - 1) / af::RED_THREADS);
    CK(c, cudaMemcpyAsync(arrays[0], c->k3[0][0], n * 8, cudaMemcpyDeviceToHost, c->stream));
    for (int a = 1; a < 8; ++a) {
      af::widen_kernel<<<grid, af::RED_THREADS, 0, c->stream>>>((const float*)c->k3[0][a], stg + a * n, n);
      CK(c, cudaGetLastError());
      CK(c, cudaMemcpyAsync(arrays[a], stg + a * n, n * 8, cudaMemcpyDeviceToHost, c->stream));
    }
  }
  CK(c, cudaStreamSynchronize(c->stream));
  return AF_OK;
}

af_status af_device_ptrs_arrays(af_ctx* c, int narr, void** ptrs, int dtype[2]) {
  if (!c || !ptrs || narr != (1 << c->dim)) return AF_E_ARG;
  if (c->dim < 3) {
    void* p4[4];
    af_status s = af_device_ptrs(c, p4, dtype);
    for (int a = 0; a < narr; ++a) ptrs[a] = p4[a];
    return s;
  }
  for (int a = 0; a < 8; ++a) ptrs[a] = c->k3[0][a];
  if (dtype) { dtype[0] = 8; dtype[1] = (int)pt_size(c); }
  return AF_OK;
}

af_status af_device_ptrs(af_ctx* c, void* ptrs[4], int dtype[2]) {
  if (!c || !ptrs) return AF_E_ARG;
  ptrs[0] = c->ub[0];
  ptrs[1] = c->pv[0];
  ptrs[2] = c->dim == 2 ? c->px[0] : nullptr;
  ptrs[3] = c->dim == 2 ? c->py[0] : nullptr;
  if (dtype) { dtype[0] = 8; dtype[1] = (int)pt_size(c); }
  return AF_OK;
}

af_status af_set_indicator(af_ctx* c, const double* s) {
  if (!c || !s) return AF_E_ARG;
  CK(c, cudaMemcpyAsync(c->s_ext, s, c->n * 8, cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->s_ext_user = nullptr;
  return AF_OK;
}

af_status af_set_indicator_device(af_ctx* c, const double* s) {
  if (!c || !s) return AF_E_ARG;
  c->s_ext_user = s;
  return AF_OK;
}

af_status af_forward_euler(af_ctx* c, double tau) {
  if (!c || !(tau >= 0.0)) return AF_E_ARG;
  if (c->bounds_pending) FAIL(c, AF_E_STATE, "state not set");
  af_status s = set_dt(c, tau, false);
  if (s != AF_OK) return s;
  if (c->dim == 3) {
    const OutSpec out = {1, 0.0, -1, 1.0, 1.0, 0};
    s = stage3d_out(c, 0, &out, 1);
    if (s != AF_OK) return s;
  } else if (c->prec == AF_PREC_FP64) {
    auto a = base_args<double>(c, 0);
    set_out<double>(c, a, 0, 1, 0.0, -1, 1.0, 1.0, 0);
    CK(c, launch<double>(c, a));
  } else {
    auto a = base_args<float>(c, 0);
    set_out<float>(c, a, 0, 1, 0.0, -1, 1.0, 1.0, 0);
    CK(c, launch<float>(c, a));
  }
  // the result goes back into buffer 0 (one copy of the state's span), so the state
  // always lives there and buffers 1.. stay the contiguous staging area of
  // af_set_state / af_get_state
  const size_t span = (size_t)((unsigned char*)c->ub[1] - (unsigned char*)c->ub[0]);
  CK(c, cudaMemcpyAsync(c->ub[0], c->ub[1], span, cudaMemcpyDeviceToDevice, c->stream));
  return AF_OK;
}

// Buffer roles. SSP-RK3 (U0..U2): U1 = FE(U0); U2 = 3/4 U0 + 1/4 FE(U1);
// U0 = 1/3 U0 + 2/3 FE(U2) (in place: U0 is only read pointwise in that stage).
// SSP-RK(5,4) (U0..U3): U1 = FE(U0); U2 = a U0 + b FE(U1); U3 = a U0 + b FE(U2);
// U1 = a U0 + b FE(U3) and U2 = a U2 + b FE(U3, own ratio); U0 = U2 + b FE(U1).
af_status af_stage(af_ctx* c, int k, double dt) {
  if (!c || !(dt >= 0.0)) return AF_E_ARG;
  if (c->bounds_pending) FAIL(c, AF_E_STATE, "state not set");
  if (k < 0 || k >= af_num_stages(c)) FAIL(c, AF_E_ARG, "stage %d out of range", k);
  if (k == 0 && dt > 0.0) {
    af_status s = set_dt(c, dt, true);
    if (s != AF_OK) return s;
  }
  return stage_any(c, k);
}

af_status af_dt_device(af_ctx* c) {
  if (!c) return AF_E_ARG;
  if (c->bounds_pending) FAIL(c, AF_E_STATE, "state not set");
  return dt_device(c, c->dt_dev, c->t_dev);
}

af_status af_step(af_ctx* c, double dt, double* dt_used) {
  if (!c || dt != dt) return AF_E_ARG;
  if (c->bounds_pending) FAIL(c, AF_E_STATE, "state not set");
  af_status s = dt > 0.0 ? set_dt(c, dt, true) : dt_device(c, c->dt_dev, c->t_dev);
  if (s != AF_OK) return s;
  for (int k = 0; k < af_num_stages(c); ++k) {
    s = stage_any(c, k);
    if (s != AF_OK) return s;
  }
  if (dt_used) return read_scalar(c, c->dt_dev, dt_used);
  return AF_OK;
}

af_status af_run(af_ctx* c, double T, long long* nsteps) {
  if (!c || !(T >= 0.0)) return AF_E_ARG;
  if (c->bounds_pending) FAIL(c, AF_E_STATE, "state not set");
  double t;
  af_status s = read_scalar(c, c->t_dev, &t);
  if (s != AF_OK) return s;
  // Steps are issued in chunks without a host round trip: the device clips each CFL
  // step to the time left before T and counts the positive ones; the steps of a chunk
  // after T is reached have dt = 0, and a stage with dt = 0 writes nothing.
  double* count = c->red + 0;   // slot 0: step count of af_run
  CK(c, cudaMemsetAsync(count, 0, sizeof(double), c->stream));
  const int chunk = 16;
  while (t < T * (1.0 - 1e-14)) {
    for (int q = 0; q < chunk; ++q) {
      s = dt_device(c, c->dt_dev, c->t_dev, T, count);
      if (s != AF_OK) return s;
      for (int k = 0; k < af_num_stages(c); ++k) {
        s = stage_any(c, k);
        if (s != AF_OK) return s;
      }
    }
    const double t_prev = t;
    s = read_scalar(c, c->t_dev, &t);
    if (s != AF_OK) return s;
    if (!(t > t_prev)) FAIL(c, AF_E_STATE, "non-positive CFL time step");
  }
  double n = 0.0;
  s = read_scalar(c, count, &n);
  if (s != AF_OK) return s;
  if (nsteps) *nsteps = (long long)n;
  long long cl = 0, er = 0;
  double mx = 0;
  s = af_stats(c, &cl, &er, &mx, nullptr);
  if (s != AF_OK) return s;
  if (er) FAIL(c, AF_E_STATE, "%lld values left [umin, umax] beyond the safeguard tolerance", er);
  return AF_OK;
}

af_status af_time(af_ctx* c, double* t) {
  if (!c || !t) return AF_E_ARG;
  return read_scalar(c, c->t_dev, t);
}

af_status af_mass(af_ctx* c, double* mass) {
  if (!c || !mass) return AF_E_ARG;
  af_status s = is_rect(c) ? reduce_array<double>(c, c->ub[0], c->pn, 0, 0.0, c->red + 1, 0, c->pnx, 1, 1)
                           : reduce_array<double>(c, c->ub[0], c->n, 0, 0.0, c->red + 1, 0);
  if (s != AF_OK) return s;
  double v;
  s = read_scalar(c, c->red + 1, &v);
  if (s != AF_OK) return s;
  *mass = v * c->dx * c->dy * c->dz;   // dz = 1 below 3D
  return AF_OK;
}

af_status af_bounds(af_ctx* c, double* umin, double* umax) {
  if (!c || !umin || !umax) return AF_E_ARG;
  if (c->dim == 3) {
    for (int op = 1; op <= 2; ++op)
      for (int a = 0; a < 8; ++a) {
        const double init = op == 1 ? INFINITY : -INFINITY;
        af_status s = (a == 0 || c->prec == AF_PREC_FP64)
                          ? reduce_array<double>(c, (const double*)c->k3[0][a], c->n, op, init, c->red + 1 + op, a > 0)
                          : reduce_array<float>(c, (const float*)c->k3[0][a], c->n, op, init, c->red + 1 + op, a > 0);
        if (s != AF_OK) return s;
      }
    af_status s = read_scalar(c, c->red + 2, umin);
    if (s != AF_OK) return s;
    return read_scalar(c, c->red + 3, umax);
  }
  const int na = c->dim == 2 ? 4 : 2;
  void* arrs[4] = {c->ub[0], c->pv[0], c->px[0], c->py[0]};
  for (int op = 1; op <= 2; ++op) {
    for (int a = 0; a < na; ++a) {
      af_status s;
      const double init = op == 1 ? INFINITY : -INFINITY;
      // DoFs of the padded rectangle: ub from (1, 1), V everywhere, X from row 1, Y from column 1
      const bool r = is_rect(c);
      const int w = r ? c->pnx : 0, ilo = r && (a == 0 || a == 3) ? 1 : 0, jlo = r && (a == 0 || a == 2) ? 1 : 0;
      const size_t cnt = r ? c->pn : (a == 0 ? c->n : c->np);
      if (a == 0 || c->prec == AF_PREC_FP64)
        s = reduce_array<double>(c, (const double*)arrs[a], cnt, op, init, c->red + 1 + op, a > 0, w, ilo, jlo);
      else
        s = reduce_array<float>(c, (const float*)arrs[a], cnt, op, init, c->red + 1 + op, a > 0, w, ilo, jlo);
      if (s != AF_OK) return s;
    }
  }
  af_status s = read_scalar(c, c->red + 2, umin);
  if (s != AF_OK) return s;
  return read_scalar(c, c->red + 3, umax);
}

af_status af_dt_cfl(af_ctx* c, double* dt) {
  if (!c || !dt) return AF_E_ARG;
  if (c->bounds_pending) FAIL(c, AF_E_STATE, "state not set");
  af_status s = dt_device(c, c->red + 4, nullptr);
  if (s != AF_OK) return s;
  return read_scalar(c, c->red + 4, dt);
}

af_status af_stats(af_ctx* c, long long* clamps, long long* errors, double* max_excess, double* mass_adjust) {
  if (!c) return AF_E_ARG;
  DevStats st;
  CK(c, cudaMemcpyAsync(&st, c->stats, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (clamps) *clamps = (long long)st.clamps;
  if (errors) *errors = (long long)st.errors;
  if (max_excess) {
    double v;
    std::memcpy(&v, &st.max_excess_bits, sizeof(v));
    *max_excess = v;
  }
  if (mass_adjust) *mass_adjust = st.ub_adjust * c->dx * c->dy * c->dz;
  return AF_OK;
}

af_status af_stats_detail(af_ctx* c, long long* avg_clamps) {
  if (!c) return AF_E_ARG;
  DevStats st;
  CK(c, cudaMemcpyAsync(&st, c->stats, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (avg_clamps) *avg_clamps = (long long)st.avg_clamps;
  return AF_OK;
}

}  // extern "C"
