"""Pins of the oracle's view-dependent colour (oracle/sh.cpp): the basis
against scipy's complex spherical harmonics, orthonormality on the sphere by
exact quadrature, closed-form colours, and the colour and end-to-end loss
gradients against central finite differences."""
import numpy as np
import pytest
from scipy.special import roots_legendre, sph_harm_y

import oracle
from datagen import GaussianSet
from datagen.scenes import with_sh
from datagen import workloads


def _dirs(n, seed):
    d = np.random.default_rng(seed).normal(size=(n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_basis_matches_scipy_real_harmonics(degree):
    """Y_l0 = Y_l^0, Y_lm = sqrt2 Re Y_l^m, Y_l,-m = sqrt2 Im Y_l^m (m > 0),
    scipy's Y_l^m carrying the Condon-Shortley phase; order m = -l..l."""
    d = _dirs(200, degree)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))      # polar
    phi = np.arctan2(d[:, 1], d[:, 0])              # azimuth
    want = []
    for l in range(1, degree + 1):
        for m in range(-l, l + 1):
            Y = sph_harm_y(l, abs(m), theta, phi)
            want.append(Y.real if m == 0 else np.sqrt(2) * (Y.real if m > 0 else Y.imag))
    np.testing.assert_allclose(oracle.sh_basis(d, degree), np.stack(want, 1), atol=1e-12)


def test_basis_is_orthonormal_on_the_sphere():
    # Gauss-Legendre in cos(theta) x uniform azimuth integrates every product
    # of two degree-3 harmonics (degree 6 polynomials) exactly
    x, wx = roots_legendre(8)
    phi = np.arange(16) * 2 * np.pi / 16
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    w = (wx[:, None] * np.full(16, 2 * np.pi / 16)[None, :]).reshape(-1)
    Y = oracle.sh_basis(d, 3)
    gram = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(15), atol=1e-12)
    # and the harmonics of degree >= 1 integrate to zero against the constant
    np.testing.assert_allclose(w @ Y, 0, atol=1e-12)


class _Cam:
    def __init__(self, t):
        self.t = np.asarray(t, np.float64)


def test_colour_closed_forms():
    g = GaussianSet(np.array([[0.0, 0.0, 2.0], [1.0, 2.0, 2.0]]), np.zeros((2, 3)),
                    np.tile([1.0, 0, 0, 0], (2, 1)), np.zeros(2),
                    np.array([[0.2, 0.3, 0.4], [0.5, 0.5, 0.5]]))
    cam = _Cam([0.0, 0.0, 0.0])
    np.testing.assert_array_equal(oracle.sh_colour(g, cam), g.rgb)    # no SH: rgb
    sh = np.zeros((2, 3, 3))
    sh[:, 1] = [0.1, -0.2, 0.3]            # l = 1, m = 0: Y = sqrt(3 / 4 pi) z
    g.sh_rest = sh
    c1 = np.sqrt(3 / (4 * np.pi))
    dz = np.array([1.0, 2.0 / 3.0])        # z of the unit directions (0,0,2)/2, (1,2,2)/3
    want = g.rgb + c1 * dz[:, None] * np.array([0.1, -0.2, 0.3])
    np.testing.assert_allclose(oracle.sh_colour(g, cam), want, atol=1e-15)
    # seen from the opposite side, Y_lm(-d) = (-1)^l Y_lm(d)
    g2 = GaussianSet(*(np.array(a) for a in g.arrays()), sh_rest=np.random.default_rng(0)
                     .normal(size=(2, 15, 3)))
    mirrored = GaussianSet(-g2.means, *(np.array(a) for a in g2.arrays()[1:]), sh_rest=g2.sh_rest)
    parity = np.array([(-1) ** l for l in range(1, 4) for _ in range(2 * l + 1)])
    c_b = oracle.sh_colour(GaussianSet(g2.means, *(np.array(a) for a in g2.arrays()[1:]),
                                       sh_rest=g2.sh_rest * parity[None, :, None]),
                           _Cam([0, 0, 0])) - g2.rgb
    np.testing.assert_allclose(oracle.sh_colour(mirrored, _Cam([0, 0, 0])) - g2.rgb, c_b,
                               atol=1e-14)
    assert np.abs(c_b).max() > 0.1


def test_colour_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    M, D = 6, 3
    g = GaussianSet(rng.normal(size=(M, 3)) + [0, 0, 3], np.zeros((M, 3)),
                    np.tile([1.0, 0, 0, 0], (M, 1)), np.zeros(M), rng.uniform(size=(M, 3)),
                    sh_rest=rng.normal(size=(M, 15, 3)))
    cam = _Cam([0.3, -0.2, 0.1])
    wgt = rng.normal(size=(M, 3))                   # L = sum wgt * c
    d_means, d_sh = np.zeros((M, 3)), np.zeros((M, 15, 3))
    lib = oracle.lib()
    P = oracle._p
    lib.orc_sh_backward(M, D, P(oracle._f64(g.means)), P(oracle._f64(g.sh_rest)), P(cam.t),
                        P(oracle._f64(wgt)), P(d_means), P(d_sh))
    h = 1e-6
    for name, grad in (("means", d_means), ("sh_rest", d_sh)):
        arr = getattr(g, name)
        for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(20)]:
            Ls = []
            for sgn in (1, -1):
                a = arr.copy()
                a[idx] += sgn * h
                gp = GaussianSet(g.means if name != "means" else a, g.log_scales, g.quats,
                                 g.opacity_logits, g.rgb,
                                 sh_rest=g.sh_rest if name != "sh_rest" else a)
                Ls.append(float((oracle.sh_colour(gp, cam) * wgt).sum()))
            fd = (Ls[0] - Ls[1]) / (2 * h)
            assert abs(fd - grad[idx]) <= 1e-7 * max(1.0, abs(fd)), (name, idx, fd, grad[idx])


def test_loss_gradient_through_sh_matches_finite_differences():
    """End to end (projection, OIT composite, L1 loss, adjoints) with degree-3
    colour: gradients of the SH coefficients and of the means, which now also
    move the viewing direction, against central differences."""
    w = workloads.grad(M=400, width=64, height=48)
    f = w.frames[0]
    g = with_sh(w.gaussians, 3, seed=5, scale=0.2).astype(np.float64)
    g.log_scales += 0.8
    rng = np.random.default_rng(4)
    Ct = np.clip(f.rgb + rng.normal(0, 0.1, size=f.rgb.shape), 0, 1).astype(np.float64)
    Dt = f.depth.astype(np.float64)
    base = oracle.render_loss_grads(g, f.cam, Ct, Dt, f.rgb, f.depth)
    vis = np.nonzero(base["rec"][:, oracle.R_VIS] > 0)[0]
    h = 1e-5
    checked = 0
    for attempt in range(300):
        if checked >= 30:
            break
        i = int(rng.choice(vis))
        name = ("sh_rest", "means")[attempt % 2]
        arr = getattr(g, name)
        idx = (i,) + tuple(int(rng.integers(0, s)) for s in arr.shape[1:])
        Ls, sig = [], []
        for sgn in (1, -1):
            a = arr.copy()
            a[idx] += sgn * h
            gp = GaussianSet(*(np.array(x) for x in g.arrays()), sh_rest=g.sh_rest.copy())
            setattr(gp, name, a)
            r = oracle.render_loss_grads(gp, f.cam, Ct, Dt, f.rgb, f.depth)
            Ls.append(r["L"])
            sig.append((r["out"]["n"].tobytes(), np.sign(r["out"]["C"] - f.rgb).tobytes()))
        ref = (base["out"]["n"].tobytes(), np.sign(base["out"]["C"] - f.rgb).tobytes())
        if sig[0] != ref or sig[1] != ref:
            continue
        fd = (Ls[0] - Ls[1]) / (2 * h)
        an = base["grads"][name][idx]
        if abs(an) < 1e-7:
            continue
        assert abs(fd - an) < 1e-4 * abs(an), (name, idx, fd, an)
        checked += 1
    assert checked >= 20, checked
