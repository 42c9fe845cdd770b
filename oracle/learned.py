"""Learned Newton initial guess (an extension of Sec. 3.2, Eq. Newton-initial-guess,
whose plain guess is S_m): the stage increment is extrapolated from the same
stage of the previous step, d_prev = u^m - S_m, and a per-element MLP, one
per SDIRK stage, trained online on converged stages, predicts the remaining
correction; the result only seeds Newton.

Definition (shared by the CUDA library, which implements it separately):
  features of element e  x_e = [u^n/s0, (u^n - u^{n-1})/s1, d_prev/s2]
      (each block [N_v][N_m] flattened, s_k[v] = per-variable RMS of the block
      over the mesh, 1 where that RMS is 0)
  network                a1 = tanh(x W1 + b1), a2 = tanh(a1 W2 + b2), y = a2 W3 + b3
  prediction             u^m_0 = S_m + d_prev + y (x) tau_m  (tau_m[v] = per-variable
                         RMS of the last training target of stage m)
  loss                   L = sum (y - T)^2 / (2 E N_v N_m),
                         T = (u^m - S_m - d_prev) / tau_m
  optimiser              Adam (lr, beta1, beta2, eps) on FP32 master parameters
Every matrix product takes BF16 operands (weights, x, a1, a2 and the output
gradients rounded to nearest-even BF16) and accumulates in FP32 on the GPU;
here the same rounding points are emulated and the products are exact FP64.
"""
import numpy as np

BF16_ROUNDING = True


def bf16(x):
    """Round to the nearest BF16 value (ties to even), via FP32."""
    if not BF16_ROUNDING:
        return np.asarray(x, dtype=np.float64)
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = (b + 0x7FFF + lsb) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def var_rms(F, nv):
    """Per-variable RMS of F [E][nv*nm] over elements and modes (1 if 0)."""
    E = F.shape[0]
    r = np.sqrt(np.mean(F.reshape(E, nv, -1) ** 2, axis=(0, 2)))
    r[r == 0] = 1.0
    return r


def features(u_hist, dprev, nv):
    """x [E][3*nv*nm] from the last two step solutions u_hist = (u^n, u^{n-1})
    and the previous increment of the stage."""
    u0, u1, d = (np.asarray(a, dtype=np.float64).reshape(a.shape[0], -1)
                 for a in (u_hist[0], u_hist[1], dprev))
    blocks = [u0, u0 - u1, d]
    out = []
    for F in blocks:
        s = var_rms(F, nv)
        out.append((F.reshape(F.shape[0], nv, -1) / s[None, :, None]).reshape(F.shape[0], -1))
    return np.concatenate(out, axis=1)


class MLP:
    """Parameters p = (W1, b1, W2, b2, W3, b3), FP32 master copies held as float64
    values that are exactly representable in FP32."""

    def __init__(self, params):
        self.p = [np.asarray(w, dtype=np.float32).astype(np.float64) for w in params]
        self.m = [np.zeros_like(w) for w in self.p]
        self.v = [np.zeros_like(w) for w in self.p]
        self.t = 0

    def forward(self, x):
        W1, b1, W2, b2, W3, b3 = self.p
        xb = bf16(x)
        z1 = xb @ bf16(W1) + b1
        a1 = np.tanh(z1)
        a1b = bf16(a1)
        z2 = a1b @ bf16(W2) + b2
        a2 = np.tanh(z2)
        a2b = bf16(a2)
        y = a2b @ bf16(W3) + b3
        return y, (xb, a1, a1b, a2, a2b)

    def loss_and_grads(self, x, T):
        """Loss and gradients with the BF16 rounding points of the GPU kernels."""
        W1, b1, W2, b2, W3, b3 = self.p
        y, (xb, a1, a1b, a2, a2b) = self.forward(x)
        n = y.size
        L = 0.5 * np.sum((y - T) ** 2) / n
        dy = (y - T) / n
        dyb = bf16(dy)
        gW3 = a2b.T @ dyb
        gb3 = dy.sum(axis=0)
        da2 = dyb @ bf16(W3).T
        dz2 = da2 * (1 - a2 * a2)
        dz2b = bf16(dz2)
        gW2 = a1b.T @ dz2b
        gb2 = dz2.sum(axis=0)
        da1 = dz2b @ bf16(W2).T
        dz1 = da1 * (1 - a1 * a1)
        dz1b = bf16(dz1)
        gW1 = xb.T @ dz1b
        gb1 = dz1.sum(axis=0)
        return L, [gW1, gb1, gW2, gb2, gW3, gb3]

    def adam(self, grads, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        """One Adam step (Kingma & Ba) on the master parameters, rounded to FP32."""
        self.t += 1
        c1 = 1 - b1 ** self.t
        c2 = 1 - b2 ** self.t
        for i, g in enumerate(grads):
            self.m[i] = b1 * self.m[i] + (1 - b1) * g
            self.v[i] = b2 * self.v[i] + (1 - b2) * g * g
            upd = lr * (self.m[i] / c1) / (np.sqrt(self.v[i] / c2) + eps)
            self.p[i] = np.asarray(self.p[i] - upd, dtype=np.float32).astype(np.float64)
