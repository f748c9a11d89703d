"""Plumbing of the autograd wrapper (PseudofermionAction) on the CPU: a fake
library object computes the action and the force with the oracle (dense LU),
and torch.autograd.gradcheck compares the wrapper's backward with finite
differences of its forward, for all terms with and without the Gaussian term
and for single Hasenbusch terms (Section 5.1, Eqs. p_dot, f_chi_i)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W  # noqa: E402
from oracle import action as oa  # noqa: E402
from oracle.lattice import Lattice as OLat  # noqa: E402
from paper_1804_07195_gb300 import _abi  # noqa: E402
from paper_1804_07195_gb300.autograd import PseudofermionAction  # noqa: E402


class OracleLibrary:
    """Stands in for a Context: action() and force() with the oracle."""

    def __init__(self, lat):
        self.lat = lat
        self.solve = oa.SolveA(lat, "dense")
        self.calls = []

    def _parts(self, phi, masses, chis, term, flags):
        p = phi.detach().numpy()
        c = [x.numpy() for x in chis]
        terms = range(len(masses) + 1) if term < 0 else [term]
        return p, c, terms, bool(flags & _abi.HMC_GAUSSIAN)

    def action(self, phi, masses, chis, term=-1, flags=0, opts=None):
        self.calls.append(("action", term, flags))
        p, c, terms, gauss = self._parts(phi, masses, chis, term, flags)
        S = sum(oa.term_action(self.lat, p, masses, c, i, self.solve) for i in terms)
        return S + (oa.gaussian_action(self.lat, p) if gauss else 0.0), {}

    def force(self, phi, masses, chis, term=-1, flags=0, opts=None):
        self.calls.append(("force", term, flags))
        p, c, terms, gauss = self._parts(phi, masses, chis, term, flags)
        g = sum(oa.term_grad(self.lat, p, masses, c, i, self.solve) for i in terms)
        if gauss:
            g = g + oa.grad_gaussian(self.lat, p)
        return torch.tensor(g), {}


@pytest.mark.parametrize("gaussian,term", [(False, -1), (True, -1), (False, 0), (False, 2)])
def test_backward_is_the_derivative_of_forward(gaussian, term):
    masses = [0.3, 1.0]
    w = W.small(2, 1, 4, seed=31, masses=masses)
    lat = OLat.from_params(w.lat)
    lib = OracleLibrary(lat)
    chis = [torch.tensor(c) for c in oa.make_chi(lat, w.phi, masses, w.rho, lib.solve)]
    phi = torch.tensor(w.phi * 0.7, requires_grad=True)
    f = lambda p: PseudofermionAction.apply(p, lib, masses, chis, None, gaussian, term)
    assert torch.autograd.gradcheck(f, (phi,), eps=1e-6, atol=1e-6, rtol=1e-5)
    flags = _abi.HMC_FERMION | (_abi.HMC_GAUSSIAN if gaussian else 0)
    assert ("force", term, flags) in lib.calls and ("action", term, flags) in lib.calls


def test_incoming_gradient_scales_the_force():
    masses = [0.5]
    w = W.small(2, 1, 4, seed=32, masses=masses)
    lat = OLat.from_params(w.lat)
    lib = OracleLibrary(lat)
    chis = [torch.tensor(c) for c in oa.make_chi(lat, w.phi, masses, w.rho, lib.solve)]
    phi = torch.tensor(w.phi, requires_grad=True)
    S = PseudofermionAction.apply(phi, lib, masses, chis)
    (3.0 * S).backward()
    ref = 3.0 * sum(oa.term_grad(lat, w.phi, masses, [c.numpy() for c in chis], i, lib.solve) for i in range(2))
    assert np.allclose(phi.grad.numpy(), ref, rtol=1e-12, atol=1e-12)
