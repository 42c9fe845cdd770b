"""Seeded random vectors (numpy PCG64) in the solution layout [E][N_v][N_m]."""
import numpy as np


def random_direction(u, seed):
    """v ~ N(0,1) per coefficient, scaled by the RMS of each variable of u."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal(u.shape)
    rms = np.sqrt(np.mean(u ** 2, axis=(0, 2)))
    rms[rms == 0] = 1.0
    return v * rms[None, :, None]


def perturbation(shape, seed, scale=0.01):
    """N(0,1)*scale samples (seeded) used to perturb an initial field."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * rng.standard_normal(shape)


def mlp_params(d_in, hidden, d_out, seed, zero_last=False):
    """Seeded initial parameters of the learned-guess MLP, FP32 values:
    W ~ N(0, 1/fan_in), b = 0 (W1 [d_in][hidden], b1, W2 [hidden][hidden], b2,
    W3 [hidden][d_out], b3); zero_last starts the output layer at 0 (the guess
    then starts as the plain extrapolation)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W1 = rng.standard_normal((d_in, hidden)) / np.sqrt(d_in)
    W2 = rng.standard_normal((hidden, hidden)) / np.sqrt(hidden)
    W3 = rng.standard_normal((hidden, d_out)) / np.sqrt(hidden)
    if zero_last:
        W3 = np.zeros_like(W3)
    out = [W1, np.zeros(hidden), W2, np.zeros(hidden), W3, np.zeros(d_out)]
    return [np.asarray(a, dtype=np.float32) for a in out]
