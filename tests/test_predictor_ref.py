"""Pins of the FP64 predictor reference (CPU only).

The reference's gradient is checked against central finite differences of
its own loss (a dropped term, a wrong tap offset or a transposed operand in
the backward pass fails this), its convolution against a per-element
brute-force sum, its bfloat16 rounding against torch's conversion, and the
masking against the invariance it promises (features beyond a protein's
length change nothing).
"""
import numpy as np
import pytest

from oracle import predictor_ref as ref

NP = sum(5 * ci * co + co for ci, co in zip(ref.CIN, ref.COUT))


def _params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    p = np.empty(NP)
    off = 0
    for ci, co in zip(ref.CIN, ref.COUT):
        p[off:off + 5 * ci * co] = rng.uniform(-1, 1, 5 * ci * co) * scale * np.sqrt(6 / (5 * ci))
        off += 5 * ci * co
        p[off:off + co] = rng.uniform(-0.1, 0.1, co)
        off += co
    return p


def _data(seed, B=2, L=9, lengths=(9, 6)):
    rng = np.random.default_rng(seed)
    f = rng.uniform(-1, 1, (B, L, 32))
    t = rng.uniform(0, 3, (B, L, 8))
    return f, t, np.array(lengths)


def test_param_count():
    assert NP == 32 * 128 * 5 + 128 + 2 * (128 * 128 * 5 + 128) + 128 * 8 * 5 + 8


def test_conv_matches_brute_force():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 7, 4))
    w = rng.normal(size=(5, 4, 3))
    z = ref._conv(x, w)
    for b in range(2):
        for l in range(7):
            for co in range(3):
                s = 0.0
                for t in range(5):
                    p = l + t - 2
                    if 0 <= p < 7:
                        s += sum(x[b, p, ci] * w[t, ci, co] for ci in range(4))
                assert abs(z[b, l, co] - s) < 1e-12


def test_gradient_matches_finite_differences():
    p = _params(11)
    f, t, ln = _data(12)
    loss, g = ref.loss_and_grad(p, f, t, ln)
    rng = np.random.default_rng(13)
    # coordinates from every layer's weights and biases
    idx, off = [], 0
    for ci, co in zip(ref.CIN, ref.COUT):
        idx += list(off + rng.integers(0, 5 * ci * co, 6))
        off += 5 * ci * co
        idx += list(off + rng.integers(0, co, 2))
        off += co
    eps = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (ref.loss_and_grad(pp, f, t, ln)[0] - ref.loss_and_grad(pm, f, t, ln)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_loss_is_mean_square_over_valid_entries():
    p = _params(5)
    f, t, ln = _data(6)
    y, _ = ref.forward(p, f, ln)
    loss, _ = ref.loss_and_grad(p, f, t, ln)
    e = [((y[b, :ln[b]] - t[b, :ln[b]]) ** 2) for b in range(len(ln))]
    assert abs(loss - np.concatenate(e).mean()) < 1e-12


def test_positions_beyond_length_change_nothing():
    p = _params(7)
    f, t, ln = _data(8)
    f2, t2 = f.copy(), t.copy()
    f2[1, ln[1]:] = 123.0
    t2[1, ln[1]:] = -7.0
    y1, _ = ref.forward(p, f, ln)
    y2, _ = ref.forward(p, f2, ln)
    assert np.array_equal(y1[1, :ln[1]], y2[1, :ln[1]])
    assert not y2[1, ln[1]:].any()
    l1, g1 = ref.loss_and_grad(p, f, t, ln)
    l2, g2 = ref.loss_and_grad(p, f2, t2, ln)
    assert l1 == l2 and np.array_equal(g1, g2)


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    x = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-6, 6, 2000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 3.0e38]])
    mine = ref.bf16_round(x)
    theirs = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mine, theirs)


def test_bf16_forward_is_close_to_fp64():
    p = _params(21)
    f, _, ln = _data(22)
    y64, _ = ref.forward(p, f, ln)
    y16, _ = ref.forward(p, f, ln, bf16=True)
    err = np.linalg.norm(y16 - y64) / np.linalg.norm(y64)
    assert 0 < err < 3e-2
