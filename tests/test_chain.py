"""Host logic of the Markov-chain driver (the HMC outline of Section 2) with a
fake context in place of the library: the heat-bath draws have the stated
distributions and count, the Metropolis step accepts with probability
min(1, exp(-dH)), a rejected trajectory leaves the field as it was, and
run_chain thermalises and measures on the stated cadence. CPU only."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1804_07195_gb300 import chain  # noqa: E402


class FakeContext:
    """Stands in for a Context: one 'trajectory' adds 1 to every entry of the
    trial field and reports the given energy change."""

    def __init__(self, N, dH):
        self.N = N
        self.dH = dH
        self.draws = []

    def md_trajectory(self, phi, pi, masses, rhos, integ, md_opts, action_opts):
        assert len(rhos) == len(masses) + 1
        self.draws.append((pi.clone(), [r.clone() for r in rhos]))
        phi.add_(1.0)
        return 0.0, self.dH, {}


def zeros(N):
    return torch.zeros(N, dtype=torch.float64)


@pytest.mark.parametrize("dH", [0.7, 2.0])
def test_acceptance_probability_is_min_1_exp_minus_dH(dH):
    ctx = FakeContext(8, dH)
    ch = chain.Chain(ctx, zeros(8), [], None, None, seed=11)
    n = 4000
    acc = sum(ch.trajectory(None)[1] for _ in range(n))
    p = math.exp(-dH)
    assert abs(acc / n - p) <= 4 * math.sqrt(p * (1 - p) / n)
    assert chain.acceptance_probability(dH) == p
    assert chain.acceptance_probability(-dH) == 1.0


def test_rejected_trajectories_keep_the_field_and_accepted_ones_take_the_trial():
    ctx = FakeContext(5, 60.0)  # exp(-60): never accepted
    ch = chain.Chain(ctx, zeros(5), [0.2], None, None, seed=3)
    for _ in range(50):
        _, a = ch.trajectory(None)
        assert not a
    assert torch.equal(ch.phi, zeros(5))
    ctx.dH = -1.0  # always accepted
    for k in range(1, 6):
        _, a = ch.trajectory(None)
        assert a
        assert torch.equal(ch.phi, torch.full((5,), float(k), dtype=torch.float64))


def test_heat_bath_draws():
    """pi ~ N(0, 1) and rho with real and imaginary parts N(0, 1/2) (weight
    exp(-rho^dagger rho)), one rho per Hasenbusch term; the same seed gives the
    same draws."""
    N = 20000
    draws = []
    for seed in (5, 5, 6):
        ctx = FakeContext(N, 0.0)
        ch = chain.Chain(ctx, zeros(N), [0.1, 0.5], None, None, seed=seed)
        ch.trajectory(None)
        draws.append(ctx.draws[0])
    pi, rhos = draws[0]
    assert len(rhos) == 3
    tol = 5 / math.sqrt(N)
    assert abs(pi.mean().item()) < tol and abs(pi.var().item() - 1.0) < 4 * tol
    for r in rhos:
        assert r.dtype == torch.complex128
        assert abs(r.real.var().item() - 0.5) < 3 * tol and abs(r.imag.var().item() - 0.5) < 3 * tol
        assert abs((r.abs() ** 2).mean().item() - 1.0) < 4 * tol
    assert torch.equal(draws[0][0], draws[1][0]) and torch.equal(draws[0][1][2], draws[1][1][2])
    assert not torch.equal(draws[0][0], draws[2][0])


def test_run_chain_thermalises_and_measures_on_its_cadence():
    ctx = FakeContext(4, -1.0)
    phi0 = zeros(4)
    seen = []
    res = chain.run_chain(ctx, phi0, 20, [], None, None, None, seed=1, therm=5,
                          measure=lambda p: seen.append(p[0].item()) or p[0].item(), measure_every=3)
    assert torch.equal(phi0, zeros(4))  # the input field is not modified
    assert res.trajectories == 20 and res.accepted == 20 and res.acceptance == 1.0
    assert len(ctx.draws) == 25
    # every trajectory is accepted and adds 1: measurements after trajectories 6, 9, ..., 24
    assert res.measurements == seen == [6.0 + 3 * k for k in range(7)]
    assert res.dH == [-1.0] * 20


class MomentumContext(FakeContext):
    """A 'trajectory' that depends on the draws: phi moves by 0.1 pi and dH is
    pi[0] (so the Metropolis decisions vary); it reports solver statistics."""

    def md_trajectory(self, phi, pi, masses, rhos, integ, md_opts, action_opts):
        phi.add_(0.1 * pi + 0.01 * rhos[0].real)
        return 1.0, 1.0 + float(pi[0]), {"iters": 7, "true_rel_res": 1e-11}


def test_checkpoint_resume_continues_the_chain_exactly(tmp_path):
    N, masses = 16, [0.3]
    full = chain.Chain(MomentumContext(N, 0.0), zeros(N), masses, None, None, seed=99)
    dh_full = [full.trajectory(None)[0] for _ in range(12)]
    part = chain.Chain(MomentumContext(N, 0.0), zeros(N), masses, None, None, seed=99)
    dh = [part.trajectory(None)[0] for _ in range(5)]
    path = str(tmp_path / "chain.npz")
    part.save(path)
    resumed = chain.Chain.load(MomentumContext(N, 0.0), path, None, None, device="cpu")
    assert resumed.masses == masses and resumed.trajectories == 5
    dh += [resumed.trajectory(None)[0] for _ in range(7)]
    assert dh == dh_full
    assert torch.equal(resumed.phi, full.phi)
    assert resumed.trajectories == full.trajectories == 12 and resumed.accepted == full.accepted
    assert 0 < full.accepted < 12


def test_run_log_has_one_json_line_per_trajectory(tmp_path):
    import json
    path = str(tmp_path / "run.jsonl")
    ch = chain.Chain(MomentumContext(8, 0.0), zeros(8), [], None, None, seed=4, log=path)
    out = [ch.trajectory(None) for _ in range(6)]
    lines = [json.loads(s) for s in open(path).read().splitlines()]
    assert [r["trajectory"] for r in lines] == list(range(1, 7))
    assert [r["dH"] for r in lines] == [d for d, _ in out]
    assert [r["accepted"] for r in lines] == [bool(a) for _, a in out]
    assert all(r["H1"] - r["H0"] == r["dH"] and r["solver"]["iters"] == 7 for r in lines)
