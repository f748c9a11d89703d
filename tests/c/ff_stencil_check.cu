// Host run of the float-float operator stencils (csrc/operator_ff.cuh) over a
// whole lattice, for comparison with the oracle (tests/test_ff_stencil.py).
// Input file: int32 n, m, nt; float64 delta, kappa, ms; float64 phi[N];
// complex128 psi[N] (canonical layout, N = 2 n m nt). Output file: complex128
// M psi, then complex128 M^dagger psi. The neighbour indices are computed here
// with plain integer arithmetic, independently of the kernels' fast division.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "operator_ff.cuh"

using namespace hmc;
using namespace hmc::ffa;

// complex128 array read as complex float-float values (the phase table and
// the input vector)
struct Table {
  const double* v;
  __host__ __device__ CFF operator()(int k) const { return cff_from(v[2 * (size_t)k], v[2 * (size_t)k + 1]); }
};

int main(int argc, char** argv) {
  if (argc != 3) {
    std::fprintf(stderr, "usage: %s in.bin out.bin\n", argv[0]);
    return 2;
  }
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  int32_t dims[3];
  double par[3];
  if (std::fread(dims, 4, 3, f) != 3 || std::fread(par, 8, 3, f) != 3) return 2;
  const int n = dims[0], m = dims[1], nt = dims[2];
  const double delta = par[0], kappa = par[1], ms = par[2];
  const int V = n * m, H = nt * V, N = 2 * H;
  std::vector<double> phi(N), psi(2 * (size_t)N);
  if (std::fread(phi.data(), 8, N, f) != (size_t)N || std::fread(psi.data(), 8, 2 * (size_t)N, f) != 2 * (size_t)N)
    return 2;
  std::fclose(f);

  std::vector<double> e(2 * (size_t)N);
  for (int k = 0; k < N; ++k) {
    e[2 * (size_t)k] = std::cos(phi[k]);
    e[2 * (size_t)k + 1] = std::sin(phi[k]);
  }
  const Table E{e.data()}, L{psi.data()};
  const FF dm = ff_from_double(delta * ms), dk = ff_from_double(delta * kappa);

  std::vector<double> outM(2 * (size_t)N), outD(2 * (size_t)N);
  auto put = [](std::vector<double>& o, int k, const CFF& v) {
    o[2 * (size_t)k] = ff_to_double(v.re);
    o[2 * (size_t)k + 1] = ff_to_double(v.im);
  };
  for (int q = 0; q < H; ++q) {
    const int t = q / V, c = q % V, j = c / n, i = c % n;
    Nbr nb;
    nb.q = q;
    nb.wrap_tm = t == 0;
    nb.wrap_tp = t == nt - 1;
    nb.tm = t == 0 ? q + (nt - 1) * V : q - V;
    nb.tp = t == nt - 1 ? q - (nt - 1) * V : q + V;
    nb.im1 = i == 0 ? q + (n - 1) : q - 1;
    nb.jm1 = j == 0 ? q + (m - 1) * n : q - n;
    nb.ip1 = i == n - 1 ? q - (n - 1) : q + 1;
    nb.jp1 = j == m - 1 ? q - (m - 1) * n : q + n;
    const PairFF a = m_pair_ff(H, nb, dm, dk, E, L);
    put(outM, q, a.a);
    put(outM, H + q, a.b);
    const PairFF d = mdag_pair_ff(H, nb, dm, dk, E, L);
    put(outD, q, d.a);
    put(outD, H + q, d.b);
  }
  FILE* g = std::fopen(argv[2], "wb");
  if (!g) return 2;
  std::fwrite(outM.data(), 8, outM.size(), g);
  std::fwrite(outD.data(), 8, outD.size(), g);
  std::fclose(g);
  return 0;
}
