// The integrators of Sections 4 and 5.2 as schedules of two updates,
//   Q(c):     phi <- phi + c pi
//   P(k, c):  pi  <- pi - c dS_k/dphi(phi)
// over any state type MDT that provides them: one chain (md.cu) or many
// chains advanced in lockstep (md_batched.cu). Level k < n is the chi_k
// Hasenbusch term, level n the Gaussian term plus chi_n, level -1 all of them.
#pragma once

#include <vector>

#include "hmc.h"
#include "trace.h"

namespace hmc {

// Nested Omelyan (Section 5.2), force first, over levels with steps[k] steps
// per trajectory; a ratio that is odd splits the inner step at its middle
// force (the two half steps of Section 5.2), recursively.
template <typename MDT>
struct Nested {
  MDT& md;
  std::vector<int> ratio;
  int L;
  double zeta;

  void inner_first(int k, double h) {
    if (k == L - 1) {
      md.Q(0.5 * h);
      return;
    }
    const int r = ratio[k + 1];
    const double hh = h / r;
    for (int i = 0; i < r / 2; ++i) step(k + 1, hh);
    if (r % 2) half_first(k + 1, hh);
  }
  void inner_second(int k, double h) {
    if (k == L - 1) {
      md.Q(0.5 * h);
      return;
    }
    const int r = ratio[k + 1];
    const double hh = h / r;
    if (r % 2) half_second(k + 1, hh);
    for (int i = 0; i < r / 2; ++i) step(k + 1, hh);
  }
  void step(int k, double h) {
    md.P(k, zeta * h);
    inner_first(k, h);
    md.P(k, (1.0 - 2.0 * zeta) * h);
    inner_second(k, h);
    md.P(k, zeta * h);
  }
  void half_first(int k, double h) {
    md.P(k, zeta * h);
    inner_first(k, h);
    md.P(k, 0.5 * (1.0 - 2.0 * zeta) * h);
  }
  void half_second(int k, double h) {
    md.P(k, 0.5 * (1.0 - 2.0 * zeta) * h);
    inner_second(k, h);
    md.P(k, zeta * h);
  }
};

// One trajectory of length tau. steps: the nested levels' steps per
// trajectory (nested Omelyan only); kind: HMC_INTEG_*. MDT also provides
// fg_kick(c, h): pi <- pi - c dS/dphi(phi - (h^2/24) dS/dphi(phi)), the
// middle kick of the force-gradient integrator (Eq. force_cal).
template <typename MDT>
void run_integrator(MDT& md, int kind, const std::vector<int>& steps, int nmd, double zeta, double tau) {
  if (kind == HMC_INTEG_NESTED_OMELYAN) {
    Nested<MDT> nest{md, {}, (int)steps.size(), zeta};
    nest.ratio.push_back(steps[0]);
    for (size_t k = 1; k < steps.size(); ++k) nest.ratio.push_back(steps[k] / steps[k - 1]);
    const double h0s = tau / steps[0];
    for (int i = 0; i < steps[0] && md.ok(); ++i) {
      HMC_TRACE("md step");
      nest.step(0, h0s);
    }
  } else if (kind == HMC_INTEG_LEAPFROG) {
    const double h = tau / nmd;
    for (int i = 0; i < nmd && md.ok(); ++i) {
      HMC_TRACE("md step");
      md.Q(0.5 * h);
      md.P(-1, h);
      md.Q(0.5 * h);
    }
  } else {
    const double h = tau / nmd;
    for (int i = 0; i < nmd && md.ok(); ++i) {
      HMC_TRACE("md step");
      md.P(-1, h / 6.0);
      md.Q(0.5 * h);
      md.fg_kick((2.0 / 3.0) * h, h);
      md.Q(0.5 * h);
      md.P(-1, h / 6.0);
    }
  }
}

}  // namespace hmc
