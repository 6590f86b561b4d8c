"""FFT lengths beyond one CTA's shared memory (global-buffer mode of the Theta and phi stages),
marked gpu.  A full-sky plan at lmax 4000 has 4L = 16000 and n_phi = 16128, both above the FP64
shared-memory limit of 14336 complex elements, so both FFT stages of the FP64 form run on global
buffers, while the FP32 form of the same points still fits shared memory.  Checked against the
oracle's direct summation at sampled points and by the adjoint identity."""
import math

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LMAX, S = 4000, 2


def _points(n=3000, seed=21):
    rng = np.random.default_rng(seed)
    th = np.arccos(rng.uniform(-1.0, 1.0, n))
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    return th, ph


def _alm(rng):
    n = O.nalm(LMAX)
    l, _ = O.lm_of_index(LMAX)
    a = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / (l + 1.0)
    return O.canonical_alm(a, LMAX, S)


@pytest.fixture(scope="module")
def case():
    from paper_2603_17166_gb300 import Plan

    th, ph = _points()
    rng = np.random.default_rng(22)
    g, c = _alm(rng), _alm(rng)
    plan = Plan(S, LMAX, torch.from_numpy(th).cuda(), torch.from_numpy(ph).cuda(), 1e-10, precision="fp64")
    return th, ph, g, c, plan


def test_plan_uses_global_buffers(case):
    th, ph, g, c, plan = case
    i = plan.info
    assert i["full_sky"] == 1
    assert i["nTheta"] > 14336 and i["nphi"] > 14336


def test_synthesis_matches_direct_sum(case):
    th, ph, g, c, plan = case
    f = plan.synthesis(torch.from_numpy(g).cuda(), torch.from_numpy(c).cuda()).cpu().numpy()
    sel = np.random.default_rng(23).choice(th.size, 48, replace=False)
    ref = O.direct_synthesis(LMAX, S, g, c, th[sel], ph[sel])
    assert O.rel_l2(f[sel], ref) <= 10 * 1e-10


def test_adjoint_identity_and_fp32_agreement(case):
    from paper_2603_17166_gb300 import Plan

    th, ph, g, c, plan = case
    rng = np.random.default_rng(24)
    f = rng.standard_normal(th.size) + 1j * rng.standard_normal(th.size)
    Aa = plan.synthesis(torch.from_numpy(g).cuda(), torch.from_numpy(c).cuda()).cpu().numpy()
    gt, ct = plan.adjoint(torch.from_numpy(f).cuda())
    gt, ct = gt.cpu().numpy(), ct.cpu().numpy()
    lhs = O.map_dot(f, Aa)
    rhs = O.alm_dot(gt, g, LMAX) + O.alm_dot(ct, c, LMAX)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    p32 = Plan(S, LMAX, torch.from_numpy(th).cuda(), torch.from_numpy(ph).cuda(), 1e-5, precision="fp32")
    assert p32.info["nphi"] <= 28672 and p32.info["nTheta"] <= 28672  # shared-memory path
    f32 = p32.synthesis(torch.from_numpy(g).cuda().to(torch.complex64),
                        torch.from_numpy(c).cuda().to(torch.complex64)).cpu().numpy()
    assert O.rel_l2(f32.astype(np.complex128), Aa) <= 10 * 1e-5
    g32, _ = p32.adjoint(torch.from_numpy(f).cuda().to(torch.complex64))
    assert O.alm_rel_l2(g32.cpu().numpy().astype(np.complex128), gt, LMAX) <= 1e-4
