"""The allocation-free entry point psht_ring_synthesis_noalloc (marked gpu).

It serves callers that cannot allocate device memory (their memory belongs to another allocator,
or they must not trigger the device-wide synchronisation cudaMalloc/cudaFree can cause).  This
file is named to run last: it calls the new entry point through the C ABI twice in a row on the
same fixed scratch array and checks both results against the planned path's ring coefficients
(psht_plan_ring_coeffs) at the same rings, within the FP64 stage-parity tolerance of the suite, and
every column |m| <= lmax against the oracle's ring synthesis (spin 0-3, rings on both sides of the
equator and on the poles).
"""
import math

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _alm(rng, lmax, s):
    n = O.nalm(lmax)
    return O.canonical_alm(rng.standard_normal(n) + 1j * rng.standard_normal(n), lmax, s)


@pytest.mark.parametrize("s,pole,radius,lmax", [(2, "N", 0.5, 400), (0, "S", 0.3, 511)])
def test_noalloc_matches_planned_ring_coefficients(s, pole, radius, lmax):
    from paper_2603_17166_gb300 import Plan, psht

    rng = np.random.default_rng(31 + s)
    th = np.arccos(rng.uniform(math.cos(radius), 1.0, 2000))
    if pole == "S":
        th = math.pi - th
    ph = rng.uniform(0, 2 * math.pi, th.size)
    plan = Plan(s, lmax, torch.from_numpy(th).cuda(), torch.from_numpy(ph).cuda(), 1e-10, precision="fp64")
    M = plan.info["M"]
    theta_j, _, _ = plan.rings()
    for call in range(2):  # two calls in a row on the shared scratch array
        g = _alm(rng, lmax, s)
        c = _alm(rng, lmax, s) if s else None
        gd = torch.from_numpy(g).cuda()
        cd = None if c is None else torch.from_numpy(c).cuda()
        ref = plan.ring_coeffs(gd, cd).cpu().numpy()                   # existing entry point
        F = psht.ring_synthesis_noalloc(s, lmax, torch.from_numpy(theta_j).cuda(), gd, cd)
        torch.cuda.synchronize()
        got = F.cpu().numpy()[:, lmax - M:lmax + M + 1]
        assert O.rel_l2(got, ref) < 1e-12, call
        # beyond the plan's phi band limit the coefficients are negligible
        assert np.abs(F.cpu().numpy()).max() < 10 * np.abs(ref).max()


@pytest.mark.parametrize("s,rings", [(2, "S"), (1, "both"), (3, "both"), (0, "N")])
def test_noalloc_full_width_against_oracle(s, rings):
    """Every column |m| <= lmax (no polar cutoff) against the oracle's ring synthesis at the same
    colatitudes, with c != 0 at spin > 0 so that the two Wigner columns differ.  "S" puts every ring
    past the equator (each evaluated by reflection), "both" mixes rings on both sides of it and the
    two poles themselves; two calls in a row share the scratch array."""
    from paper_2603_17166_gb300 import psht

    rng = np.random.default_rng(57 + s)
    lmax = 300
    if rings == "S":
        th = math.pi - np.linspace(0.02, 0.6, 37)
    elif rings == "both":
        th = np.concatenate([[0.0, math.pi, 0.5 * math.pi], rng.uniform(0.0, math.pi, 60)])
    else:
        th = np.linspace(0.0, 0.9, 29)
    for call in range(2):
        g = _alm(rng, lmax, s)
        c = _alm(rng, lmax, s) if s else None
        F = psht.ring_synthesis_noalloc(s, lmax, torch.from_numpy(th).cuda(), torch.from_numpy(g).cuda(),
                                        None if c is None else torch.from_numpy(c).cuda())
        torch.cuda.synchronize()
        got = F.cpu().numpy()
        ref = O.ring_synthesis(lmax, s, lmax, g, c, th)
        assert got.shape == ref.shape
        assert O.rel_l2(got, ref) < 1e-12, call
        # per ring, and against the largest value (columns beyond the turning point are tiny)
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 1e-12 * scale * lmax
        for j in range(th.size):
            if np.linalg.norm(ref[j]) > 1e-6 * np.linalg.norm(ref):
                assert O.rel_l2(got[j], ref[j]) < 1e-11, (call, j)


def test_noalloc_checks_buffer_sizes_on_the_host():
    """The C entry point takes no buffer sizes; the binding checks them before any device work, so
    a short a_lm array or a wrongly shaped output raises ValueError instead of reaching the GPU."""
    from paper_2603_17166_gb300 import psht

    lmax = 16
    th = torch.linspace(0.1, 0.5, 5, dtype=torch.float64, device="cuda")
    g = torch.zeros(O.nalm(lmax), dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError):
        psht.ring_synthesis_noalloc(0, lmax, th, g[:-1])
    with pytest.raises(ValueError):
        psht.ring_synthesis_noalloc(2, lmax, th, g, g[:-3])
    with pytest.raises(ValueError):
        psht.ring_synthesis_noalloc(0, lmax, th, g, out=torch.empty((5, 2 * lmax), dtype=torch.complex128,
                                                                      device="cuda"))
    with pytest.raises(ValueError):
        psht.ring_synthesis_noalloc(0, lmax, th, g, out=torch.empty((5, 2 * lmax + 1), dtype=torch.complex64,
                                                                      device="cuda"))
    with pytest.raises(ValueError):
        psht.ring_synthesis_noalloc(0, lmax, th.reshape(5, 1), g)
    F = psht.ring_synthesis_noalloc(0, lmax, th, g)
    torch.cuda.synchronize()
    assert F.shape == (5, 2 * lmax + 1) and float(F.abs().max()) == 0.0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2603_17166_gb300 import PshtError, psht

    th = torch.zeros(4, dtype=torch.float64, device="cuda")
    g = torch.zeros(O.nalm(600), dtype=torch.complex128, device="cuda")
    with pytest.raises(PshtError):
        psht.ring_synthesis_noalloc(0, 600, th, g)
    g = torch.zeros(O.nalm(8), dtype=torch.complex128, device="cuda")
    with pytest.raises(PshtError):
        psht.ring_synthesis_noalloc(0, 8, torch.zeros(5000, dtype=torch.float64, device="cuda"), g)
    assert psht.lib().psht_noalloc_scratch_bytes() < 8 << 20
