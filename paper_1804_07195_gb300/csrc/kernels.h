// Host-side launchers of the libhmc kernels (kernels.cu). Every launcher
// enqueues on ctx->stream and returns a status; none synchronises.
#pragma once

#include <functional>

#include "ctx.h"

namespace hmc {

template <typename R>
using V2 = typename Vec2<R>::type;

// Phase tables: E = e^{i phi} (complex128) and phi rounded to float.
hmc_status k_phase_launch(hmc_ctx* c, const double* phi);

// out = M^dagger p, out = M u + sigma y (y may be NULL).
template <typename R>
hmc_status mdag_launch(hmc_ctx* c, const Geo& g, R dm, const V2<R>* p, V2<R>* out);
template <typename R>
hmc_status m_launch(hmc_ctx* c, const Geo& g, R dm, const V2<R>* u, const V2<R>* y, R sigma,
                    V2<R>* out);

// out = (M M^dagger + sigma) in in one pass, u = M^dagger in kept on chip
// (fused.cu); the tile shape is tuned on the first call per precision.
template <typename R>
hmc_status mmdag_fused_launch(hmc_ctx* c, const Geo& g, R dm, R sigma, const V2<R>* in, V2<R>* out);
FusedShape make_fused_shape(const Geo& g, int Ti, int Tj, int Tt, int D, int pairs);
template <typename R>
bool fused_ok(const Geo& g, const FusedShape& fs);
// Pin the fused kernel's tile, prefetch depth D (2 or 6) and, for FP32, the
// two-cells-per-thread kernel (pairs) for prec 32 or 64; HMC_ERR_INVALID if
// it does not fit.
hmc_status set_fused_shape(hmc_ctx* c, int prec, int Ti, int Tj, int Tt, int D, int pairs);

// Single-reduction FP32 CG (cg32_fused.cu): one launch per iteration over
// tiles of the fused M M^dagger kernel. Buffers: r, w, s alternate between
// two vectors (r[0] is the solve's residual vector), the partials between
// partA and partB.
struct CG1Bufs {
  float2* r[2];
  float2* w[2];
  float2* s[2];
  float2* part[2];
};
// Workspace vectors of the buffers (r[1] == nullptr when one cannot be had).
CG1Bufs cg1_bufs(hmc_ctx* c, float2* r0);
bool cg1_ok(const hmc_ctx* c, const Geo& g, const FusedShape& fs);
// w_0 = A r_0 and the partials of gamma_0, delta_0 (after the CG state was initialised)
hmc_status cg1_prime_launch(hmc_ctx* c, const Geo& g, const CG1Bufs& B, float2* p, float2* x, CGScal* sc);
// iteration with state slot par (successive iterations alternate 0, 1)
hmc_status cg1_iter_launch(hmc_ctx* c, const Geo& g, const CG1Bufs& B, float2* p, float2* x, CGScal* sc, int par);
// Tile tuner; reinit re-initialises the CG state before each candidate.
bool cg1_tune(hmc_ctx* c, const Geo& g, const CG1Bufs& B, float2* p, float2* x, CGScal* sc,
              const std::function<hmc_status()>& reinit);
hmc_status set_cg1_shape(hmc_ctx* c, int Ti, int Tj, int Tt, int D);

// Resident-tile FP32 CG (cg32_resident.cu): the whole solve in one
// cooperative launch with p and M^dagger p of each block's tile in shared
// memory; false / HMC_ERR_INVALID when the tiles do not fit on chip.
bool cg32_resident_ok(const hmc_ctx* c, const Geo& g);
hmc_status cg32_resident_launch(hmc_ctx* c, const Geo& g, float2* x, float2* r, float2* p0, float2* p1, float2* u,
                                CGScal* sc);

// CG building blocks on the state sc (see common.cuh).
template <typename R>
hmc_status cg_mdag_launch(hmc_ctx* c, const Geo& g, const V2<R>* p, V2<R>* u, CGScal* sc,
                          unsigned* ticket);
template <typename R>
hmc_status cg_m_launch(hmc_ctx* c, const Geo& g, const V2<R>* u, const V2<R>* p, V2<R>* x,
                       V2<R>* r, CGScal* sc, unsigned* ticket);
template <typename R>
hmc_status cg_p_launch(hmc_ctx* c, int N, const V2<R>* r, V2<R>* p, const CGScal* sc);

// FP32 CG, two kernels per iteration: p_new = r + beta p_old folded into
// u = M^dagger p_new (with pAp and alpha), then the M kernel with the updates.
// One cell-time per thread.
hmc_status cg32_pmdag_launch(hmc_ctx* c, const Geo& g, const float2* r, const float2* pold,
                             float2* pnew, float2* u, CGScal* sc, unsigned* ticket);
hmc_status cg32_m_launch(hmc_ctx* c, const Geo& g, const float2* u, const float2* p, float2* x,
                         float2* r, CGScal* sc, unsigned* ticket);

// r = b - (M u + sigma x), with |r|^2 and |b|^2 reduced. When init != NULL the
// last block initialises a CG state (rr, bb, thresh = tol2 * bb, iter 0, done if
// rr <= thresh, the operator's sigma and ddm = delta m_s) and p = r is written.
// When out2 != NULL it receives {|r|^2, |b|^2}.
template <typename R>
hmc_status resid_launch(hmc_ctx* c, const Geo& g, R dm, const V2<R>* u, const V2<R>* x,
                        const V2<R>* b, double sigma, V2<R>* r, V2<R>* p, CGScal* init,
                        double tol2, int maxit, double* out2, unsigned* ticket, double ddm = 0.0);

// x = 0, r = p = b, |b|^2 reduced into a fresh CG state (with sigma, ddm).
template <typename R>
hmc_status init0_launch(hmc_ctx* c, int N, const V2<R>* b, V2<R>* x, V2<R>* r, V2<R>* p, CGScal* sc,
                        double tol2, int maxit, double sigma, unsigned* ticket, double ddm);

// Whether the shared-memory tiled FP32 CG kernels apply to this lattice at
// `tc` cells and `tt` time slices per tile.
bool cg32_tiled_ok(const hmc_ctx* c, const Geo& g, int tc, int tt);
// Whether the marching FP32 CG kernels' reduction partials fit their buffers
// at `threads` cells and `tt` time slices per block.
bool cg32_march_ok(const hmc_ctx* c, const Geo& g, int threads, int tt);
// Launch (no instrumentation) of the tiled or marching kernels of the pair
// for the shape sh; GB / GA: the other kernel's partial count.
void cg32_alt_pmdag(hmc_ctx* c, const Geo& g, const Shape& sh, const float2* r, const float2* pold, float2* pnew,
                    float2* u, CGScal* sc, int GB);
void cg32_alt_m(hmc_ctx* c, const Geo& g, const Shape& sh, const float2* u, const float2* p, float2* x, float2* r,
                CGScal* sc, int GA);
// The persistent FP32 CG kernel: whether its on-chip state fits this lattice,
// and one cooperative launch that runs the whole solve from the state k_init0
// (or the residual kernel) left in sc, x, r and p0 (p1: second direction
// buffer, u: scratch).
bool cg32_persist_ok(const hmc_ctx* c, const Geo& g);
// The last launch of a CG loop body: sets the loop condition (sc still
// running and fewer trips than loop_trips[1]) and counts the trip.
hmc_status loop_continue_launch(hmc_ctx* c, cudaGraphConditionalHandle h, const CGScal* sc);
hmc_status cg32_persist_launch(hmc_ctx* c, const Geo& g, float2* x, float2* r, float2* p0, float2* p1,
                               float2* u, CGScal* sc);

// Resident blocks per SM of a CG kernel at `threads` threads per block
// (pairs: the FP32 kernels with two cells per thread).
int cg_kernel_occupancy(int id, int threads, int pairs = 0);

// Precision conversions.
hmc_status to32_launch(hmc_ctx* c, int N, const double2* in, float2* out);
hmc_status to64_launch(hmc_ctx* c, int N, const float2* in, double2* out);

// |v|^2 into *out (device).
hmc_status norm2_launch(hmc_ctx* c, int N, const double2* v, double* out, unsigned* ticket);

// FGMRES pieces (Algorithm A.1), all FP64:
//   mdot:  h[i] = V_i^H w, i < nv (complex, written to hout as 2*nv doubles)
//   gsupd: w -= sum_i h[i] V_i, then |w|^2 into *ww
//   scale: v = s w and v32 = (float) v
//   xupd:  x += sum_i y[i] Z_i
constexpr int kMaxRestart = 16;
struct VecList {
  const double2* v[kMaxRestart];
};
struct CoefList {
  double re[kMaxRestart], im[kMaxRestart];
};
hmc_status mdot_launch(hmc_ctx* c, int N, VecList V, int nv, const double2* w, double* hout,
                       unsigned* ticket);
hmc_status gsupd_launch(hmc_ctx* c, int N, VecList V, int nv, const double* h, double2* w,
                        double* ww, unsigned* ticket);
hmc_status scale_launch(hmc_ctx* c, int N, double s, const double2* w, double2* v, float2* v32);
hmc_status xupd_launch(hmc_ctx* c, int N, VecList Z, CoefList y, int nz, double2* x);

// y = a x + y (real vectors) and y = a x + b y (complex128).
hmc_status axpy_real_launch(hmc_ctx* c, int N, double a, const double* x, double* y);
hmc_status axpby_c_launch(hmc_ctx* c, int N, double a, const double2* x, double b, double2* y);

// Force of one pseudofermion term (Eqs. f_chi_i / p_dot), accumulated:
//   g[k] += -2 Re( conj(eta[k]) dM_k w[tp(k)] ),  w = xi - chi (chi may be NULL).
hmc_status force_launch(hmc_ctx* c, const Geo& g, const double2* eta, const double2* xi,
                        const double2* chi, double* grad);
// g[k] (+)= phi[k] / (delta U)
hmc_status gauss_grad_launch(hmc_ctx* c, int N, const double* phi, double inv_dU, int accumulate,
                             double* grad);
// *out = sum phi^2 / 2 * scale_phi + sum pi^2 / 2 (pi may be NULL), deterministic.
hmc_status half_sq_launch(hmc_ctx* c, int N, const double* a, double sa, const double* b, double* out,
                          unsigned* ticket);
// *out = Re(u^H v) (deterministic)
hmc_status redot_launch(hmc_ctx* c, int N, const double2* u, const double2* v, double* out,
                        unsigned* ticket);

}  // namespace hmc
