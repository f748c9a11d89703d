// out = (M M^dagger + sigma) in, complex128, for callers that cannot allocate
// device memory: no context, no cudaMalloc, no library allocation (the
// operator of Eq. ferm_op, in FP64).
//
// The intermediate M^dagger in lives in a file-scope static device array of
// HMC_NOALLOC_MAX_SITES complex128 entries (16 MiB), which every GPU that loads
// this library keeps until the process exits. The phases e^{i phi} are
// computed inline from phi (no phase table). The array's host-side name is
// not a device address, so its device address is looked up once per device
// with cudaGetSymbolAddress, under a lock, on that device's first call.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "hmc.h"
#include "operator.cuh"
#include "validate.h"

namespace hmc {
namespace {

__device__ __align__(256) double2 g_noalloc_u[HMC_NOALLOC_MAX_SITES];

// e^{i phi_k} from phi itself (FP64 sine and cosine).
struct PhaseSincos {
  const double* phi;
  __device__ __forceinline__ Cx<double> operator()(int k) const {
    double s, c;
    sincos(phi[k], &s, &c);
    return Cx<double>{c, s};
  }
};

__global__ void __launch_bounds__(256) kn_mdag(Geo g, PhaseSincos ph, double dm,
                                               const double2* __restrict__ in, double2* __restrict__ u) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < g.H; q += gridDim.x * blockDim.x) {
    Nbr nb = neighbours(g, q);
    PairOut<double> o = mdag_pair<double, PhaseSincos>(g, ph, dm, in, nb);
    st(u, q, o.a);
    st(u, g.H + q, o.b);
  }
}

__global__ void __launch_bounds__(256) kn_m(Geo g, PhaseSincos ph, double dm, const double2* __restrict__ u,
                                            const double2* __restrict__ in, double sigma,
                                            double2* __restrict__ out) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < g.H; q += gridDim.x * blockDim.x) {
    Nbr nb = neighbours(g, q);
    PairOut<double> o = m_pair<double, PhaseSincos>(g, ph, dm, u, nb);
    double2 ya = in[q], yb = in[g.H + q];
    o.a.re = fma(sigma, ya.x, o.a.re);
    o.a.im = fma(sigma, ya.y, o.a.im);
    o.b.re = fma(sigma, yb.x, o.b.re);
    o.b.im = fma(sigma, yb.y, o.b.im);
    st(out, q, o.a);
    st(out, g.H + q, o.b);
  }
}

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double2* g_scratch[kMaxDevices] = {};

}  // namespace
}  // namespace hmc

using namespace hmc;

extern "C" hmc_status hmc_apply_MMdag_noalloc(const hmc_lattice* lat, const double* phi, double ms,
                                              double sigma, const void* in, void* out, void* cuda_stream) {
  // every check runs before the first CUDA call: a rejected call touches no device
  if (bad_lattice(lat)) return HMC_ERR_INVALID;  // the same checks as hmc_create
  if (!phi || !in || !out) return HMC_ERR_INVALID;
  const long long N = lattice_sites(lat);
  if (((uintptr_t)phi) % 8 || ((uintptr_t)in) % 16 || ((uintptr_t)out) % 16) return HMC_ERR_INVALID;
  if (ranges_overlap(in, out, (size_t)N * sizeof(double2))) return HMC_ERR_INVALID;
  if (!(sigma >= 0.0) || !std::isfinite(sigma) || !std::isfinite(ms)) return HMC_ERR_INVALID;
  const double delta = lat->beta / lat->nt;
  if (1.0 - delta * ms == 0.0) return HMC_ERR_INVALID;
  if (N > (long long)HMC_NOALLOC_MAX_SITES) return HMC_ERR_NOMEM;  // beyond the static scratch

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return HMC_ERR_CUDA;
  }
  double2* u = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_u) != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return HMC_ERR_CUDA;
      }
      g_scratch[dev] = (double2*)p;
    }
    u = g_scratch[dev];
  }
  const Geo g = make_geo(lat->n, lat->m, lat->nt, delta, lat->kappa);
  const PhaseSincos ph{phi};
  const double dm = delta * ms;
  const int threads = 256;
  const int grid = (int)((g.H + threads - 1) / threads);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  kn_mdag<<<grid, threads, 0, s>>>(g, ph, dm, (const double2*)in, u);
  kn_m<<<grid, threads, 0, s>>>(g, ph, dm, u, (const double2*)in, sigma, (double2*)out);
  if (cudaGetLastError() != cudaSuccess) return HMC_ERR_CUDA;
  return HMC_OK;
}
