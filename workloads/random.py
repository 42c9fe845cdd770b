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
