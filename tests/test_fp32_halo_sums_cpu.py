"""The arithmetic the FP32 form's AT halo kernel uses, emulated on the host with the library's own
AT weight tables: why the sums over the delayed levels' differences need compensation.

Each stage value is S U_0 + sum_{l>=1} W_l (U_l - U_0) (Eq. 14-15; the weights of a stage sum to
S = 1).  For long delays the weights alternate in sign with sum |W| up to about 1,400, so
rounding the differences U_l - U_0 to FP32 and summing them plainly multiplies their rounding by
that factor.  With the differences and weights as exact float pairs and the products summed by
TwoSum, the result has the accuracy of the FP64 sum before its final rounding to FP32.  No GPU:
float32 arithmetic is emulated with numpy (an FMA as the exact FP64 product of two floats plus the
addend, rounded once to float32)."""
import numpy as np
import pytest

from paper_2506_03027_gb300 import build as B
from paper_2506_03027_gb300 import cfs

f32 = np.float32


@pytest.fixture(scope="module")
def weights():
    B.build()
    cfs.load()
    return cfs.cfs_at_weights(4, 4)  # [k][m][l], LSERK4-CD4-AT4, delays 0..4


def _levels(k, n, slope, rng):
    """n smooth histories U(t) = b + s t + c t^2 sampled at the delayed levels t = -(k + l)."""
    b = rng.uniform(0.5, 2.0, n) * rng.choice([-1.0, 1.0], n)
    s = rng.uniform(-slope, slope, n)
    c = rng.uniform(-slope / 10, slope / 10, n)
    t = -(k + np.arange(5.0))
    return b[:, None] + s[:, None] * t + c[:, None] * t * t, np.abs(b)


def _trunc32(x):
    """FP32 truncation toward zero of FP64 values, and the rest rounded once to FP32."""
    h = x.astype(f32)
    over = np.abs(h.astype(np.float64)) > np.abs(x)
    h = np.where(over, np.nextafter(h, f32(0)), h)
    return h, (x - h.astype(np.float64)).astype(f32)


def _fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def _plain(W, r):
    """FP32 differences rounded once, plain FP32 sums."""
    h0 = r[:, 0].astype(f32)
    l0 = (r[:, 0] - h0.astype(np.float64)).astype(f32)
    a = (r[:, 1:] - r[:, :1]).astype(f32)
    out = []
    for m in range(W.shape[0]):
        d = f32(W[m].sum() - 1.0) * h0
        for l in range(1, 5):
            d = (d + f32(W[m, l]) * a[:, l - 1]).astype(f32)
        out.append(h0 + (l0 + d))
    return np.stack(out, 1)


def _compensated(W, r):
    """Exact float pairs for the differences and the weights, products split with an FMA, TwoSum."""
    h0 = r[:, 0].astype(f32)
    l0 = (r[:, 0] - h0.astype(np.float64)).astype(f32)
    ah, al = [], []
    for l in range(1, 5):
        h, q = _trunc32(r[:, l])
        ah.append(h - h0)
        al.append(q - l0)
    out = []
    for m in range(W.shape[0]):
        sh = np.zeros_like(h0)
        st = f32(W[m].sum() - 1.0) * h0
        for l in range(1, 5):
            wh = f32(W[m, l])
            wl = f32(W[m, l] - np.float64(wh))
            p = wh * ah[l - 1]
            pe = _fma32(np.full_like(p, wh), ah[l - 1], -p)
            s2 = sh + p
            bv = s2 - sh
            se = (sh - (s2 - bv)) + (p - bv)
            sh = s2
            st = st + (se + pe)
            st = _fma32(np.full_like(p, wh), al[l - 1], st)
            st = _fma32(np.full_like(p, wl), ah[l - 1], st)
        out.append(h0 + (l0 + (sh + st)))
    return np.stack(out, 1)


def _errors(W, k, slope, seed=0, n=4000):
    rng = np.random.default_rng(seed)
    r, scale = _levels(k, n, slope, rng)
    exact = r @ W[k].T                                  # FP64 sums, every stage
    ref = exact.astype(f32)                             # what the FP64 sums gave after rounding
    e = lambda v: np.mean(np.abs(v.astype(np.float64) - exact).max(1) / scale)
    return e(ref), e(_plain(W[k], r)), e(_compensated(W[k], r))


def test_weights_of_every_stage_sum_to_one(weights):
    assert np.abs(weights.sum(-1) - 1.0).max() < 1e-12
    assert np.abs(weights[4]).sum(-1).max() > 1000     # the amplification of long delays


@pytest.mark.parametrize("k", [0, 2, 4])
def test_compensated_sums_match_the_fp64_sums(weights, k):
    """Per-level changes of 1 % of the value (coarse grids at large CFL): the compensated sums lose
    nothing against the FP64 sums rounded to FP32; plain FP32 sums lose the weights' amplification
    at long delays."""
    e_ref, e_plain, e_comp = _errors(weights, k, 1e-2)
    assert e_comp < 1.1 * e_ref, (e_ref, e_comp)
    if k == 4:
        assert e_plain > 5 * e_ref, (e_ref, e_plain)


def test_small_changes_do_not_need_the_compensation_but_keep_it_exact(weights):
    """With per-level changes of 5e-4 (the 256^3 benchmark's step) even plain sums stay near the
    FP32 rounding at k = 4; the compensated ones match the FP64 sums."""
    e_ref, e_plain, e_comp = _errors(weights, 4, 5e-4)
    assert e_comp < 1.1 * e_ref and e_plain < 2 * e_ref, (e_ref, e_plain, e_comp)
