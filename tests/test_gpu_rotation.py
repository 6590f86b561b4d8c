"""Rotation of a_lm, of points and the patch-centred frame through the C ABI (marked gpu), against
the oracle's plain definitions: the D-matrix sum for every coefficient at band limits that span
several output blocks with a ragged last one, selected coefficients at lmax 4096, R^-1 R = 1 at
full size, points and spin-basis angles, and the smallest enclosing cap."""
import math

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _alm(rng, lmax, s=0):
    n = O.nalm(lmax)
    return O.canonical_alm(rng.standard_normal(n) + 1j * rng.standard_normal(n), lmax, s)


ANGLES = [(0.7, 1.1, -2.4), (2.0, 2.9, 0.3), (-1.0, 0.2, 5.0), (0.3, math.pi, -0.8), (1.4, 0.0, 0.6)]


@pytest.mark.parametrize("lmax", [0, 1, 5, 64, 600])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_rotate_alm_parity(lmax, prec):
    from paper_2603_17166_gb300 import Rotator

    rng = np.random.default_rng(100 + lmax)
    g, c = _alm(rng, lmax), _alm(rng, lmax)
    rot = Rotator(lmax, precision=prec)
    # FP64: rounding of a recurrence of <= lmax steps; FP32: at most 1e-5, a tenth of the error
    # budget 10 eps of the FP32 form's smallest eps
    tol = 1e-12 if prec == "fp64" else 1e-5
    for k, ang in enumerate(ANGLES):
        gg = torch.from_numpy(g).cuda()
        cc = torch.from_numpy(c).cuda()
        go, co = rot.apply(gg, cc if k % 2 == 0 else None, *ang)
        ref_g = O.rotate_alm(lmax, g, *ang)
        assert O.alm_rel_l2(go.cpu().numpy().astype(np.complex128), ref_g, lmax) <= tol, (ang, prec)
        if k % 2 == 0:
            ref_c = O.rotate_alm(lmax, c, *ang)
            assert O.alm_rel_l2(co.cpu().numpy().astype(np.complex128), ref_c, lmax) <= tol
        _, m = O.lm_of_index(lmax)
        assert np.all(go.cpu().numpy()[m == 0].imag == 0)


def test_rotate_alm_in_place_and_one_shot():
    from paper_2603_17166_gb300 import Rotator, rotate_alm

    rng = np.random.default_rng(7)
    lmax = 77
    g = _alm(rng, lmax)
    ang = (0.4, 1.9, -0.2)
    ref = O.rotate_alm(lmax, g, *ang)
    rot = Rotator(lmax)
    t = torch.from_numpy(g).cuda()
    rot.apply(t, None, *ang, g_out=t)
    assert O.alm_rel_l2(t.cpu().numpy(), ref, lmax) <= 1e-12
    go, _ = rotate_alm(torch.from_numpy(g).cuda(), None, *ang)
    assert O.alm_rel_l2(go.cpu().numpy(), ref, lmax) <= 1e-12


@pytest.mark.parametrize("prec,tol", [("fp32", 3e-5), ("fp64", 1e-11)])
def test_rotate_alm_full_size(prec, tol):
    """lmax 4096 (the headline band limit): selected coefficients against the oracle's O(l^2) sums,
    and the inverse rotation returns the input."""
    from paper_2603_17166_gb300 import Rotator

    lmax = 4096
    rng = np.random.default_rng(8)
    n = O.nalm(lmax)
    l_all, m_all = O.lm_of_index(lmax)
    g = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / (l_all + 1.0)
    g[m_all == 0] = g[m_all == 0].real
    rot = Rotator(lmax, precision=prec)
    ang = (0.9, 0.61, -2.2)
    t = torch.from_numpy(g).cuda()
    go, _ = rot.apply(t, None, *ang)
    got = go.cpu().numpy().astype(np.complex128)
    ls = np.array([4096, 4096, 4096, 4000, 2048, 3000, 1, 4096])
    ms = np.array([0, 1, 4096, 2500, 2048, 17, 1, 3001])
    ref = O.rotate_alm_lm(lmax, g, *ang, ls, ms)
    idx = O.alm_index(lmax, ls, ms)
    # each coefficient against the rms size of its degree
    scale = np.array([np.sqrt(np.mean(np.abs(g[l_all == l]) ** 2)) for l in ls])
    assert np.all(np.abs(got[idx] - ref) <= tol * scale), (np.abs(got[idx] - ref) / scale)
    back, _ = rot.apply(go, None, -ang[2], -ang[1], -ang[0])
    assert O.alm_rel_l2(back.cpu().numpy().astype(np.complex128), g, lmax) <= 2 * tol


def test_rotate_points_parity():
    from paper_2603_17166_gb300 import rotate_points

    rng = np.random.default_rng(9)
    th = np.concatenate([np.arccos(rng.uniform(-1, 1, 5000)), [0.0, math.pi, 1e-9]])
    ph = np.concatenate([rng.uniform(-3, 9, 5000), [0.0, 1.0, 2.0]])
    for ang in ANGLES:
        t2, p2, psi = rotate_points(torch.from_numpy(th).cuda(), torch.from_numpy(ph).cuda(), *ang)
        rt, rp, rpsi = O.rotate_points(*ang, th, ph)
        t2, p2, psi = t2.cpu().numpy(), p2.cpu().numpy(), psi.cpu().numpy()
        assert np.abs(t2 - rt).max() < 1e-12
        # azimuth and basis angle are undefined where a point lands on a pole
        ok = np.sin(rt) > 1e-6
        dphi = np.angle(np.exp(1j * (p2 - rp)))
        assert np.abs(dphi[ok]).max() < 1e-12
        dpsi = np.angle(np.exp(1j * (psi - rpsi)))
        ok2 = ok & (np.sin(th) > 1e-6)
        assert np.abs(dpsi[ok2]).max() < 1e-10
        assert np.all((p2 >= 0) & (p2 < 2 * math.pi))


def test_patch_rotation_small_set_matches_oracle_cap():
    from paper_2603_17166_gb300 import patch_rotation, rotate_points

    rng = np.random.default_rng(11)
    # a box in RA/dec around dec -56 deg (colatitude ~146 deg), 300 points
    ra = rng.uniform(-0.8, 0.8, 300)
    dec = np.arcsin(rng.uniform(math.sin(math.radians(-70)), math.sin(math.radians(-42)), 300))
    th, ph = math.pi / 2 - dec, np.mod(ra, 2 * math.pi)
    eul, ts = patch_rotation(torch.from_numpy(th).cuda(), torch.from_numpy(ph).cuda())
    tc, pc, rad = O.min_enclosing_cap(th, ph)
    assert abs(ts - rad) < 1e-7
    assert abs(eul[1] - tc) < 1e-5 and abs(np.angle(np.exp(1j * (math.pi - eul[2] - pc)))) < 1e-4
    t2, _, _ = rotate_points(torch.from_numpy(th).cuda(), torch.from_numpy(ph).cuda(), *eul, want_psi=False)
    assert t2.max().item() <= ts + 1e-12


def test_patch_rotation_full_box():
    """The ~4 % RA/dec box (1' grid with deflections, 5.6e6 points, as given near the south pole):
    every point lies within the returned radius of the centre, no subsample has a larger smallest
    cap, and the radius is the ~34.7 deg of the patch-centred frame."""
    from paper_2603_17166_gb300 import patch_rotation, rotate_points
    from paper_2603_17166_gb300 import synthetic as S

    th, ph = S.field_points("grid4", "S", S.rng(2, "points"), S.rng(2, "deflections"), step_arcmin=1.0)
    th, ph = torch.from_numpy(th).cuda(), torch.from_numpy(ph).cuda()
    eul, ts = patch_rotation(th, ph)
    t2, _, _ = rotate_points(th, ph, *eul, want_psi=False)
    assert t2.max().item() <= ts + 1e-12
    sel = np.random.default_rng(12).choice(th.numel(), 250, replace=False)
    _, _, rad = O.min_enclosing_cap(th.cpu().numpy()[sel], ph.cpu().numpy()[sel])
    assert rad <= ts + 1e-9
    assert math.radians(33.0) < ts < math.radians(36.0)


def test_patch_rotation_rejects_invalid_points():
    from paper_2603_17166_gb300 import PshtError, patch_rotation

    th = torch.tensor([0.5, float("nan"), 0.7], dtype=torch.float64, device="cuda")
    ph = torch.tensor([0.1, 0.2, 0.3], dtype=torch.float64, device="cuda")
    with pytest.raises(PshtError):
        patch_rotation(th, ph)
    with pytest.raises(PshtError):
        patch_rotation(torch.tensor([0.5, 4.0], dtype=torch.float64, device="cuda"), ph[:2])
    # points not in any open hemisphere (both poles)
    with pytest.raises(PshtError):
        patch_rotation(torch.tensor([0.0, math.pi], dtype=torch.float64, device="cuda"), ph[:2])
