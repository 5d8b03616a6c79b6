"""FP64 oracle of the learned single-scatter surrogate (test infrastructure).

This module is test infrastructure: only the test suite, the smoke check and
the benchmark's CPU-baseline leg may import it.  It shares no code with the
CUDA library.

The network maps 32 inputs to one output through three hidden layers of
width 128 with the tanh form of GELU:

    z1 = W1 x + b1,  h1 = gelu(z1)
    z2 = W2 h1 + b2, h2 = gelu(z2)
    z3 = W3 h2 + b3, h3 = gelu(z3)
    out = w4 . h3 + b4

and is trained on the weighted mean squared error (1/n) sum_i v_i
(out_i - t_i)^2 with Adam (Kingma and Ba, 2015: beta1 0.9, beta2 0.999, eps
1e-8, bias-corrected moments).  The target t of one (event, voxel, line) is
ln(S_w + 1e-8), S_w the single-scatter part of the row for line w (the
n = 1 paths of Eq. (s_p) summed over the scatter points, times the detector
response); the weights v = (S_w + 1e-8)^power / mean count each sample by its
share of the scatter mass.  ``features`` restates the network's inputs from
their definition: the geometry of the voxel, the detector angle, the bin and
the recorded energy, the optical depths along eight directions, and the
scatter point p* on the bin's projection line at the scattering angle that
Compton's relation gives for the recorded energy.

Parameter vector (FP32 in the library, FP64 here), in this order:
W1[128][32], b1[128], W2[128][128], b2[128], W3[128][128], b3[128], w4[128], b4.

Parity status and pins (tests/test_oracle_mlp.py):
  gelu, gelu_grad   - odd-part identity gelu(z) - gelu(-z) = z, limits,
                      distance to the erf form, central differences
  forward/gradient  - central finite differences of the loss in FP64 on
                      every parameter block, zero gradient at an exact fit,
                      the output-bias gradient in closed form
  adam_step         - the first step from zero moments moves every
                      parameter by lr |g| / (|g| + eps) against g
  init_params       - the published SplitMix64 generator (Steele, Lea and
                      Flood, 2014) checked against its reference outputs
  scatter_reach     - the oracle's exact single-scatter sum of a line just
                      outside the range is below 1e-9 of its value inside
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 32, 128
OFF_W1 = 0
OFF_B1 = OFF_W1 + N_HID * N_IN
OFF_W2 = OFF_B1 + N_HID
OFF_B2 = OFF_W2 + N_HID * N_HID
OFF_W3 = OFF_B2 + N_HID
OFF_B3 = OFF_W3 + N_HID * N_HID
OFF_W4 = OFF_B3 + N_HID
OFF_B4 = OFF_W4 + N_HID
N_PARAMS = OFF_B4 + 1
EPS_TARGET = 1e-8

_C = np.sqrt(2.0 / np.pi)
_MASK = (1 << 64) - 1


def unpack(p):
    """Views (W1, b1, W2, b2, W3, b3, w4, b4) of the parameter vector."""
    p = np.asarray(p, dtype=np.float64)
    return (p[OFF_W1:OFF_B1].reshape(N_HID, N_IN), p[OFF_B1:OFF_W2],
            p[OFF_W2:OFF_B2].reshape(N_HID, N_HID), p[OFF_B2:OFF_W3],
            p[OFF_W3:OFF_B3].reshape(N_HID, N_HID), p[OFF_B3:OFF_W4],
            p[OFF_W4:OFF_B4], p[OFF_B4])


def pack(W1, b1, W2, b2, W3, b3, w4, b4):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, np.ravel(W3), b3, w4,
                           np.atleast_1d(b4)]).astype(np.float64)


def gelu(z):
    """0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))."""
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * z * (1.0 + np.tanh(_C * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    """d gelu / dz of the tanh form."""
    z = np.asarray(z, dtype=np.float64)
    t = np.tanh(_C * (z + 0.044715 * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * _C * (1.0 + 3.0 * 0.044715 * z * z)


def forward(p, x, keep=False):
    """Outputs [n] for inputs x [n, 32]; with keep, also the pre-activations."""
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = gelu(z2)
    z3 = h2 @ W3.T + b3
    h3 = gelu(z3)
    out = h3 @ w4 + b4
    if keep:
        return out, (x, z1, h1, z2, h2, z3, h3)
    return out


def loss(p, x, t, v=None):
    """(1/n) sum_i v_i (out_i - t_i)^2 (v = 1 when None)."""
    d = forward(p, x) - np.asarray(t, dtype=np.float64)
    v = 1.0 if v is None else np.asarray(v, dtype=np.float64)
    return float(np.mean(v * d * d))


def train_weights(t, power):
    """Sample weights exp(power (t_i - max t)), normalised to mean 1: with
    t = ln(S + eps) they count each sample by (S + eps)^power."""
    t = np.asarray(t, dtype=np.float64)
    v = np.exp(power * (t - t.max()))
    return v * (t.size / v.sum())


def gradient(p, x, t, v=None):
    """(dL/dp, L) for L = (1/n) sum_i v_i (out_i - t_i)^2, by the chain rule."""
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(p)
    out, (x, z1, h1, z2, h2, z3, h3) = forward(p, x, keep=True)
    n = x.shape[0]
    r = out - np.asarray(t, dtype=np.float64)
    v = np.ones(n) if v is None else np.asarray(v, dtype=np.float64)
    dout = 2.0 * v * r / n                     # dL/dout_i
    g_w4 = h3.T @ dout
    g_b4 = dout.sum()
    dz3 = np.outer(dout, w4) * gelu_grad(z3)   # dL/dz3
    g_W3 = dz3.T @ h2
    g_b3 = dz3.sum(axis=0)
    dz2 = (dz3 @ W3) * gelu_grad(z2)
    g_W2 = dz2.T @ h1
    g_b2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * gelu_grad(z1)
    g_W1 = dz1.T @ x
    g_b1 = dz1.sum(axis=0)
    return pack(g_W1, g_b1, g_W2, g_b2, g_W3, g_b3, g_w4, g_b4), float(np.mean(v * r * r))


def adam_step(p, m1, m2, g, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (p, m1, m2)."""
    m1 = beta1 * m1 + (1.0 - beta1) * g
    m2 = beta2 * m2 + (1.0 - beta2) * g * g
    mhat = m1 / (1.0 - beta1 ** step)
    vhat = m2 / (1.0 - beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m1, m2


def splitmix64(state: int):
    """SplitMix64: advance the state by the golden gamma and mix it.
    Returns (output, new state)."""
    state = (state + 0x9E3779B97F4A7C15) & _MASK
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31), state


def init_params(seed: int) -> np.ndarray:
    """The library's initial parameters as float32: Xavier-uniform weights
    U(-l, l), l = sqrt(6 / (fan_in + fan_out)) computed in float32, drawn in
    parameter order W1, W2, W3, w4 from one SplitMix64 stream of `seed`
    (u = top 53 bits / 2^53, value = (2u - 1) l rounded to float32); zero
    biases; output bias -10."""
    p = np.zeros(N_PARAMS, dtype=np.float32)
    state = seed & _MASK

    def fill(off, count, fan_in, fan_out):
        nonlocal state
        lim = float(np.sqrt(np.float32(6.0) / np.float32(fan_in + fan_out), dtype=np.float32))
        for i in range(count):
            z, state = splitmix64(state)
            u = (z >> 11) * (1.0 / 9007199254740992.0)
            p[off + i] = np.float32((2.0 * u - 1.0) * lim)

    fill(OFF_W1, N_HID * N_IN, N_IN, N_HID)
    fill(OFF_W2, N_HID * N_HID, N_HID, N_HID)
    fill(OFF_W3, N_HID * N_HID, N_HID, N_HID)
    fill(OFF_W4, N_HID, N_HID, 1)
    p[OFF_B4] = -10.0
    return p


ELECTRON_REST_KEV = 510.99895


def compton_kappa(e_hat, e_line):
    """1 - cos(phi) of the single scatter that takes e_line to e_hat
    (Compton: 1/E' - 1/E = (1 - cos phi) / m_e c^2)."""
    return ELECTRON_REST_KEV * (1.0 / e_hat - 1.0 / e_line)


def scatter_reach(e_line, fwhm_frac, e_ref, exponent, n_sigma=8.0):
    """(lo, hi): the recorded energies that one Compton scatter of a photon of
    energy e_line can produce, widened by n_sigma energy-resolution sigmas.
    A single scatter gives E' between the backscatter energy
    e_line / (1 + 2 e_line / m_e c^2) and e_line; the detector blurs E' with a
    Gaussian of FWHM = fwhm_frac E (E / e_ref)^exponent.  The surrogate's
    scatter part of line w is zero outside (lo, hi)."""
    def sigma(e):
        return fwhm_frac * e * (e / e_ref) ** exponent / (2.0 * np.sqrt(2.0 * np.log(2.0)))
    e_back = e_line / (1.0 + 2.0 * e_line / ELECTRON_REST_KEV)
    return e_back - n_sigma * sigma(e_back), e_line + n_sigma * sigma(e_line)


def features(x, y, theta, u_b, e_hat, w, e_line, optical_depth8, rho_map, pixel_cm):
    """The 32 inputs of one (event, voxel, line), FP64.

    x, y: voxel centre (cm); theta: detector angle; u_b: bin centre on the
    detector axis (cm); optical_depth8: mu_w(E_w) x rho-integral (cm) from
    the voxel to the image edge along theta + k pi/4, k = 0..7; rho_map:
    [n, n] density, row iy, column ix, pixel centres at
    ((i + 0.5 - n/2) h)."""
    n = rho_map.shape[0]
    ca, sa = np.cos(theta), np.sin(theta)
    f = np.zeros(32)
    f[0], f[1], f[2], f[3], f[4] = x * 0.05, y * 0.05, ca, sa, u_b * 0.05
    f[5] = (e_hat - 150.0) * 0.01
    f[6 + w] = 1.0
    f[9:17] = np.asarray(optical_depth8) * 0.25
    uq, tq = -x * sa + y * ca, x * ca + y * sa      # detector coordinate, depth
    du = u_b - uq
    kappa = compton_kappa(e_hat, e_line)
    f[17], f[18] = du * 0.2, tq * 0.05
    f[19] = min(max(kappa, -2.0), 4.0) * 0.5
    f[20], f[21] = e_hat / e_line, abs(du) * 0.2
    c = min(max(1.0 - kappa, -1.0), 1.0)           # cos(phi)
    s = max(np.sqrt(max(1.0 - c * c, 0.0)), 0.05)
    lim = n * pixel_cm
    dt = min(max(abs(du) * c / s, -lim), lim)      # p* - q along the depth axis
    tp = tq + dt
    xp, yp = tp * ca - u_b * sa, tp * sa + u_b * ca
    r = np.hypot(dt, du)
    f[22], f[23], f[24] = xp * 0.05, yp * 0.05, r * 0.05
    f[25], f[26] = c, pixel_cm / (r + pixel_cm)
    f[27] = 1.0 if kappa < 0 else 0.0
    gx, gy = np.floor(xp / pixel_cm + 0.5 * n), np.floor(yp / pixel_cm + 0.5 * n)
    f[28] = rho_map[int(gy), int(gx)] if (0 <= gx < n and 0 <= gy < n) else 0.0
    return f
