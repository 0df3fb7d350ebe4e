"""Pins of the oracle's Fourier neural operator: central finite differences
of the loss against the analytic gradients, the truncated DFT against numpy's
FFT, and Adam against its closed form on a quadratic."""
import numpy as np
import pytest

from oracle import fno

NZ, NX, MODES, W, L = 8, 6, 2, 3, 2


def _problem(seed=0):
    rng = np.random.default_rng(seed)
    p = fno.init_params(W, MODES, L, seed)
    for k in p:   # nonzero biases so their gradients are exercised
        if k.startswith("b") or k in ("p", "q"):
            p[k] = (rng.standard_normal(p[k].shape) + 1j * rng.standard_normal(p[k].shape)) * 0.3
    x = rng.standard_normal((2, NZ, NX)) + 1j * rng.standard_normal((2, NZ, NX))
    t = rng.standard_normal((NZ, NX)) + 1j * rng.standard_normal((NZ, NX))
    return p, x, t


def test_truncated_dft_matches_fft():
    rng = np.random.default_rng(1)
    v = rng.standard_normal((NZ, NX)) + 1j * rng.standard_normal((NZ, NX))
    full = np.fft.fft2(v)
    kz, kx = fno.mode_index(NZ, MODES), fno.mode_index(NX, MODES)
    part = fno.dft_rows(NZ, MODES) @ v @ fno.dft_rows(NX, MODES).T
    assert np.allclose(part, full[np.ix_(kz, kx)], atol=1e-12)


def test_spectral_layer_with_all_modes_is_circular_convolution():
    """With every mode kept and a scalar weight per mode, K is the circular
    convolution whose kernel has that DFT."""
    n = 8
    rng = np.random.default_rng(2)
    v = rng.standard_normal((1, n, n)) + 1j * rng.standard_normal((1, n, n))
    Rk = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    R = np.zeros((n, n, 1, 1), complex)
    kk = fno.mode_index(n, n // 2)
    R[:, :, 0, 0] = Rk[np.ix_(kk, kk)]
    out, _ = fno._spectral(v, R, n, n, n // 2)
    ref = np.fft.ifft2(np.fft.fft2(v[0]) * Rk)
    assert np.allclose(out[0], ref, atol=1e-12)


def test_gradients_match_central_differences():
    p, x, t = _problem()
    loss, g = fno.loss_and_grad(p, x, t, NZ, NX, MODES)
    rng = np.random.default_rng(3)
    h = 1e-6
    for name in p:
        w = p[name]
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in w.shape)
            for part, unit in (("re", 1.0), ("im", 1j)):
                w0 = w[idx]
                w[idx] = w0 + h * unit
                lp = fno.loss_and_grad(p, x, t, NZ, NX, MODES)[0]
                w[idx] = w0 - h * unit
                lm = fno.loss_and_grad(p, x, t, NZ, NX, MODES)[0]
                w[idx] = w0
                fd = (lp - lm) / (2 * h)
                an = g[name][idx].real if part == "re" else g[name][idx].imag
                assert fd == pytest.approx(an, rel=1e-6, abs=1e-9), (name, idx, part)


def test_zero_projection_is_the_identity():
    """With Q = 0 and q = 0 the output is the residual channel itself."""
    p, x, _ = _problem(5)
    p["Q"][:] = 0
    p["q"][:] = 0
    assert np.array_equal(fno.forward(p, x, NZ, NX, MODES), x[0])


def test_input_gradient_chain_through_lift():
    """The lift's input gradient, checked through P's gradient formula."""
    p, x, t = _problem(4)
    loss, g = fno.loss_and_grad(p, x, t, NZ, NX, MODES)
    assert np.isfinite(loss) and all(np.all(np.isfinite(v)) for v in g.values())


def test_adam_one_step_closed_form():
    p = {"w": np.array([1.0 + 2.0j])}
    g = {"w": np.array([0.5 - 0.25j])}
    st = {}
    fno.adam_step(p, g, st, lr=0.1)
    # first step: m_hat = g, v_hat = g^2 per part -> step = sign(g) * |g| / (|g| + eps)
    assert p["w"][0].real == pytest.approx(1.0 - 0.1 * 0.5 / (0.5 + 1e-8))
    assert p["w"][0].imag == pytest.approx(2.0 + 0.1 * 0.25 / (0.25 + 1e-8))


def test_training_reduces_loss_on_a_fixed_batch():
    p, x, t = _problem(5)
    st = {}
    l0 = fno.loss_and_grad(p, x, t, NZ, NX, MODES)[0]
    for _ in range(60):
        loss, g = fno.loss_and_grad(p, x, t, NZ, NX, MODES)
        fno.adam_step(p, g, st, lr=3e-2)
    assert loss < 0.5 * l0
