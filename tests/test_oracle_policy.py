"""Pins of the policy-network oracle (§4.1) to facts outside itself: the
output sizes that the stated kernels and strides fix, a hand-computed
receptive field, a different library routine (scipy's correlate2d) for the
convolution, brute-force loops on a tiny case, closed forms for the heads
and for categorical sampling, and torch's bfloat16 rounding."""
import numpy as np
import pytest

from oracle import policy as P
from paper_2510_01764_gb300 import workloads as W


def test_layer_sizes_follow_from_kernels_and_strides():
    """§4.1: (8,4)/(4,2), 4/2, 3/1 on the (4, 64, 32) stack."""
    sizes = [(64, 32)]
    for _, _, (kx, ky), (sx, sy) in P.CONV_SPECS:
        X, Y = sizes[-1]
        sizes.append((P.conv_out(X, kx, sx), P.conv_out(Y, ky, sy)))
    assert sizes == [(64, 32), (15, 15), (6, 6), (4, 4)]
    params = W.policy_params(1, 5)
    obs = np.zeros((2, 4, 32, 64), np.uint8)
    logits, value, acts = P.forward(params, obs, features=True)
    assert [a.shape for a in acts] == [(2, 32, 15, 15), (2, 64, 6, 6), (2, 64, 4, 4)]
    assert logits.shape == (2, 5) and value.shape == (2,)


def test_orientation_and_receptive_field_by_hand():
    """One lit pixel (frame 2, x = 9, y = 5) under conv1 weights that encode
    their own offsets: output (i, j) sees it at offset (9 - 4i, 5 - 2j) when
    that lies inside the 8 x 4 kernel, i.e. at i in {1, 2}, j in {1, 2}."""
    obs = np.zeros((1, 4, 32, 64), np.uint8)
    obs[0, 2, 5, 9] = 1                       # [frame, y, x]
    x = P.to_paper_orientation(obs)
    assert x[0, 2, 9, 5] == 1 and x.sum() == 1
    w = np.zeros((32, 4, 8, 4))
    u, v = np.meshgrid(np.arange(8), np.arange(4), indexing="ij")
    w[3, 2] = 100 * u + v + 1
    out = P.conv2d_valid(x, w, np.zeros(32), (4, 2))
    want = np.zeros((15, 15))
    want[1, 1], want[1, 2], want[2, 1], want[2, 2] = 504, 502, 104, 102
    assert np.array_equal(out[0, 3], want)
    assert not np.delete(out[0], 3, axis=0).any()


def test_conv_matches_scipy_correlate():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(3)
    for (C, O, (kx, ky), (sx, sy)), (X, Y) in zip(P.CONV_SPECS, [(64, 32), (15, 15), (6, 6)]):
        x = rng.standard_normal((2, C, X, Y))
        w = rng.standard_normal((O, C, kx, ky))
        b = rng.standard_normal(O)
        got = P.conv2d_valid(x, w, b, (sx, sy))
        for n in range(2):
            for o in range(0, O, 7):
                full = sum(signal.correlate2d(x[n, c], w[o, c], mode="valid") for c in range(C))
                np.testing.assert_allclose(got[n, o], full[::sx, ::sy] + b[o], rtol=1e-10, atol=1e-10)


def test_conv_brute_force_tiny():
    rng = np.random.default_rng(4)
    x = rng.integers(-3, 4, (1, 2, 9, 7)).astype(np.float64)
    w = rng.integers(-2, 3, (3, 2, 3, 2)).astype(np.float64)
    b = np.array([1.0, -2.0, 0.5])
    got = P.conv2d_valid(x, w, b, (2, 1))
    assert got.shape == (1, 3, 4, 6)
    for o in range(3):
        for i in range(4):
            for j in range(6):
                s = b[o]
                for c in range(2):
                    for u in range(3):
                        for v in range(2):
                            s += w[o, c, u, v] * x[0, c, 2 * i + u, j + v]
                assert got[0, o, i, j] == s


def test_heads_closed_form_with_silent_features():
    """With zero convolution weights and biases the features are 0, so the
    logits are wa2 relu(ba1) + ba2 and the value wc2 . relu(bc1) + bc2."""
    p = W.policy_params(2, 17)
    for k in ("w1", "b1", "w2", "b2", "w3", "b3"):
        p[k] = np.zeros_like(p[k])
    obs = np.random.default_rng(0).integers(0, 2, (3, 4, 32, 64)).astype(np.uint8)
    logits, value = P.forward(p, obs)
    la = p["wa2"].astype(np.float64) @ np.maximum(p["ba1"].astype(np.float64), 0) + p["ba2"]
    vc = p["wc2"].astype(np.float64) @ np.maximum(p["bc1"].astype(np.float64), 0) + p["bc2"][0]
    np.testing.assert_allclose(logits, np.tile(la, (3, 1)), rtol=1e-12)
    np.testing.assert_allclose(value, np.full(3, vc), rtol=1e-12)


def test_flatten_order_is_channel_x_y():
    """Feature index c * 16 + x * 4 + y: a head weight on one index reads
    exactly that conv3 output."""
    p = W.policy_params(5, 3)
    obs = np.random.default_rng(1).integers(0, 2, (2, 4, 32, 64)).astype(np.uint8)
    _, _, acts = P.forward(p, obs, features=True)
    c, x, y = 37, 2, 3
    q = dict(p)
    q["wc1"] = np.zeros_like(p["wc1"])
    q["wc1"][0, c * 16 + x * 4 + y] = 1.0
    q["bc1"] = np.zeros_like(p["bc1"])
    q["wc2"] = np.zeros_like(p["wc2"])
    q["wc2"][0] = 1.0
    q["bc2"] = np.zeros(1, np.float32)
    _, v = P.forward(q, obs)
    np.testing.assert_allclose(v, acts[2][:, c, x, y], rtol=1e-12)


def test_bf16_rounding_against_torch_and_by_hand():
    torch = pytest.importorskip("torch")
    one = 1.0
    assert P.bf16_round(np.array([one + 2 ** -8]))[0] == 1.0                      # tie -> even
    assert P.bf16_round(np.array([one + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6        # tie -> even
    assert P.bf16_round(np.array([one + 2 ** -8 + 2 ** -12]))[0] == 1.0 + 2 ** -7
    x = np.random.default_rng(9).standard_normal(100000).astype(np.float32) * 7
    t = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(P.bf16_round(x), t)


def test_sampling_closed_forms():
    rng = np.random.default_rng(5)
    u = rng.random(20000)
    # equal logits: a = floor(u * L)
    L = 5
    a = P.sample(np.zeros((u.size, L)), u)
    assert np.array_equal(a, np.minimum(np.floor(u * L), L - 1).astype(np.uint8))
    # one dominant logit
    lg = np.full((u.size, 4), -1e9)
    lg[:, 2] = 0.0
    assert (P.sample(lg, u) == 2).all()
    # frequencies follow softmax (chi-square, 3 degrees of freedom)
    lg = np.tile(np.array([0.0, 1.0, -0.5, 0.3]), (u.size, 1))
    p = np.exp(lg[0]) / np.exp(lg[0]).sum()
    counts = np.bincount(P.sample(lg, u), minlength=4)
    chi2 = ((counts - p * u.size) ** 2 / (p * u.size)).sum()
    assert chi2 < 16.3          # p = 0.001 for 3 degrees of freedom
    w = np.array([0, 255, 256, 0xFFFFFFFF], dtype=np.uint64)
    assert np.array_equal(P.uniform_from_word(w), [0.0, 0.0, 2.0 ** -24, 1 - 2.0 ** -24])


def test_bf16_storage_stays_close_to_float64():
    """The bfloat16-storage forward (the kernels' storage precision) differs
    from the float64 forward by a few per cent of the output scale at most."""
    p = W.policy_params(7, 5)
    obs = (np.random.default_rng(2).random((16, 4, 32, 64)) < 0.1).astype(np.uint8)
    l64, v64 = P.forward(p, obs)
    l16, v16 = P.forward(p, obs, storage="bf16")
    scale = max(1.0, float(np.sqrt((l64 ** 2).mean())))
    assert np.abs(l16 - l64).max() < 0.03 * scale
    assert np.abs(v16 - v64).max() < 0.03 * max(1.0, float(np.abs(v64).max()))
    assert np.abs(l16 - l64).max() > 0      # the rounding is really applied


def test_bf16_storage_rounds_exactly_the_tensor_core_operands():
    """Only the convolution and hidden-layer weights are rounded: changing
    an output-layer weight by less than a bfloat16 ulp still moves the
    logits, changing a conv1 weight that little does not."""
    p = W.policy_params(11, 5)
    obs = (np.random.default_rng(3).random((4, 4, 32, 64)) < 0.2).astype(np.uint8)
    base, _ = P.forward(p, obs, storage="bf16")
    q = dict(p)
    q["wa2"] = p["wa2"] * np.float32(1 + 2 ** -12)
    moved, _ = P.forward(q, obs, storage="bf16")
    assert np.abs(moved - base).max() > 0
    q = dict(p)
    w1 = P.bf16_round(p["w1"]).astype(np.float32)
    q["w1"] = w1 * np.float32(1 + 2 ** -12)          # rounds back to the same bfloat16
    assert np.array_equal(P.bf16_round(q["w1"]), P.bf16_round(w1))
    p2 = dict(p)
    p2["w1"] = w1
    same, _ = P.forward(q, obs, storage="bf16")
    ref, _ = P.forward(p2, obs, storage="bf16")
    assert np.array_equal(same, ref)
