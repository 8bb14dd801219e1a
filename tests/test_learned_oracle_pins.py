"""Pins of the learned-halo oracle pieces (CPU only): the numpy FP64 backprop against finite
differences, the C forward against numpy, and the BF16 rounding against its definition."""
import numpy as np
import pytest

from oracle import mlp
from oracle import oracle as orc


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = mlp.init_params(5).astype(np.float64)
    X = rng.standard_normal((7, mlp.NIN))
    T = rng.standard_normal((7, mlp.NOUT))
    loss, g = mlp.loss_and_grad(p, X, T)
    idx = rng.choice(mlp.NPARAM, size=40, replace=False)
    for i in idx:
        h = 1e-6
        pp = p.copy(); pp[i] += h
        pm = p.copy(); pm[i] -= h
        fd = (mlp.loss_and_grad(pp, X, T)[0] - mlp.loss_and_grad(pm, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_gelu_derivative_matches_finite_differences():
    z = np.linspace(-4, 4, 41)
    fd = (mlp.gelu(z + 1e-6) - mlp.gelu(z - 1e-6)) / 2e-6
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, rtol=1e-7, atol=1e-9)


def test_c_forward_matches_numpy():
    rng = np.random.default_rng(4)
    p = mlp.init_params(2)
    for _ in range(5):
        x = np.array([orc.bf16(v) for v in rng.standard_normal(mlp.NIN)])
        np.testing.assert_allclose(orc.mlp_forward_c(p, x), mlp.forward(p, x[None])[0][0], rtol=1e-13, atol=1e-13)


def test_bf16_rounding_is_round_to_nearest_even():
    assert orc.bf16(1.0 + 2.0 ** -8) == 1.0                    # tie -> even
    assert orc.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6     # tie -> even (upwards)
    assert orc.bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert orc.bf16(-3.0) == -3.0
    assert orc.bf16(1e-30) > 0
    x = np.random.default_rng(1).standard_normal(1000)
    for v in x:
        b = orc.bf16(v)
        assert abs(b - v) <= 2.0 ** -8 * abs(v)                  # within half a BF16 ulp


def _lagrange_at_zero(nodes):
    """Textbook Lagrange basis weights evaluating at t = 0 from samples at the given times."""
    w = []
    for i, ti in enumerate(nodes):
        num, den = 1.0, 1.0
        for j, tj in enumerate(nodes):
            if j != i:
                num *= -tj
                den *= ti - tj
        w.append(num / den)
    return w


def _levels_for_column(case, column):
    """Four full states U^t = base + c_t g (c = 7, 3, 2, 0 for t = n, n-k, n-k-1, n-k-2) with
    g = 1 + y' + 8 v + 64 [x' off the column] + 128 [z' off the column] (y' the coordinate along
    the face normal, x', z' the tangential ones): level differences are g, 2 g and 4 g -- at most
    8 significant bits, so exact in BF16 after power-of-two scales -- and every point of the
    column is identified by its value."""
    from paper_2506_03027_gb300 import inputs as I
    Z, Y, X = np.meshgrid(np.arange(case.nz), np.arange(case.ny), np.arange(case.nx), indexing="ij")
    C = (X, Y, Z)
    a, t1c, t2c = column  # normal axis, and the global coordinates along (a+1)%3, (a+2)%3
    on1 = C[(a + 1) % 3] == t1c
    on2 = C[(a + 2) % 3] == t2c
    g = np.stack([1.0 + C[a] + 8 * v + 64 * (~on1) + 128 * (~on2) for v in range(5)])
    base = 1000.0 + np.arange(5)[:, None, None, None] + np.zeros_like(g)
    return [base + ct * g for ct in (7.0, 3.0, 2.0, 0.0)], g


@pytest.mark.parametrize("face,sub,t1,t2,k,column,halo_pts,own_pts", [
    # sub-domain 5 of a 2x2x2 split of 8^3 (offset x 4, y 0, z 4), face -y: tangential axes z (t1)
    # and x (t2); local (t1, t2) = (3, 1) is global z = 7, x = 5.  Halo points beyond the -y face
    # at depths 1..4: global y = 7, 6, 5, 4 (periodic wrap); own points at depths 1..4: y = 0..3.
    (2, 5, 3, 1, 2, (1, 7, 5), [7, 6, 5, 4], [0, 1, 2, 3]),
    # the same sub-domain's +x face: tangential axes y (t1) and z (t2); local (2, 0) is global
    # y = 2, z = 4.  Halo beyond +x (local x 4..7 -> global 8..11 -> 0..3), own x = 7, 6, 5, 4.
    (1, 5, 2, 0, 4, (0, 2, 4), [0, 1, 2, 3], [7, 6, 5, 4]),
    # sub-domain 0, -z face: tangential x (t1), y (t2); halo z = 7..4, own z = 0..3; delay 0.
    (4, 0, 1, 3, 0, (2, 1, 3), [7, 6, 5, 4], [0, 1, 2, 3]),
])
def test_column_features_hand_computed(face, sub, t1, t2, k, column, halo_pts, own_pts):
    """The learned halo's features of one column (x[0..19] the level difference n-k minus n-k-1
    at the 4 halo points, x[20..39] n-k-1 minus n-k-2 there, x[40..59] n minus n-k at the 4 own
    points next to the face, x[60..64] the one-hot delay, each times its scale; index
    (depth - 1) * 5 + v) and the 3-level extrapolation of Eq. 14, against values written out for
    hand-picked columns."""
    from paper_2506_03027_gb300 import inputs as I
    case = I.tgv_case(8, 2, "SA", filter=False)
    levels, g = _levels_for_column(case, column)
    in_s = [2.0 ** -3, 2.0 ** -2, 0.5, 1.0, 2.0]
    own_s = [2.0 ** -4, 2.0 ** -5, 2.0 ** -6, 0.25, 1.0]
    scales = np.array(in_s + own_s + [1.0] * 5)
    x, at3 = orc.column_features(case, levels, scales, sub, face, t1, t2, k)
    a = column[0]

    def pt(normal):
        c = [0, 0, 0]
        c[a], c[(a + 1) % 3], c[(a + 2) % 3] = normal, column[1], column[2]
        return c[2], c[1], c[0]  # (z, y, x) index

    c3 = _lagrange_at_zero([-k, -k - 1, -k - 2])
    for j in range(4):
        zh, yh, xh = pt(halo_pts[j])
        zo, yo, xo = pt(own_pts[j])
        for v in range(5):
            gh = 1 + halo_pts[j] + 8 * v   # g on the column: no off-column terms
            go = 1 + own_pts[j] + 8 * v
            assert g[v, zh, yh, xh] == gh and g[v, zo, yo, xo] == go
            assert x[j * 5 + v] == gh * in_s[v]
            assert x[20 + j * 5 + v] == 2 * gh * in_s[v]
            assert x[40 + j * 5 + v] == 4 * go * own_s[v]
            lv = [1000.0 + v + ct * gh for ct in (3.0, 2.0, 0.0)]
            assert abs(at3[j * 5 + v] - sum(w * u for w, u in zip(c3, lv))) < 1e-10
    assert list(x[60:65]) == [1.0 if q == k else 0.0 for q in range(5)]
