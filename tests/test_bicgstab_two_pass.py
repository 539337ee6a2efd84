"""The two-pass arrangement of BiCGStab used for the Gram solves, checked on CPU.

The GPU solver forms, per iteration k, first K1 (finish step k-1 row by row:
s = r - alpha v, r_k = s - omega t, x += alpha p + omega s; then p_k and
v_k = G p_k) and then K2 (s_k = r_k - alpha_k v_k, t_k = G s_k), taking
rho_k = r0^H r_k from the K2 sums as r0^H s - omega r0^H t. This test writes
that arrangement in numpy and compares its iterates with the textbook
arrangement (van der Vorst 1992) on small random complex systems with a real
well-conditioned matrix, as the Gram systems are. No CUDA code is involved.
"""
import numpy as np


def textbook(G, b, iters):
    x = np.zeros_like(b)
    r = b.copy()
    rh = b.copy()
    rho_prev = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    xs = []
    for _ in range(iters):
        rho = np.vdot(rh, r)
        beta = (rho / rho_prev) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = G @ p
        alpha = rho / np.vdot(rh, v)
        s = r - alpha * v
        t = G @ s
        omega = np.vdot(t, s) / np.vdot(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_prev = rho
        xs.append(x.copy())
    return xs


def two_pass(G, b, iters):
    """K1 of iteration k finishes step k-1; rho from the K2 sums."""
    x = np.zeros_like(b)
    r_prev = b.copy()          # r_{-1} = b with zero scalars gives r_0 = b, p_0 = b
    rh = b.copy()
    p_prev = np.zeros_like(b)
    v_prev = np.zeros_like(b)
    t = np.zeros_like(b)
    alpha = omega = beta = 0.0
    rho = np.vdot(b, b)
    xs = []
    sums = None
    for k in range(iters + 1):
        # K1: scalars from the previous K2 sums
        if k > 0:
            ts, tt, r0s, r0t = sums
            omega = ts / tt
            rho_new = r0s - omega * r0t
            beta = (rho_new / rho) * (alpha / omega)
            rho = rho_new
        s = r_prev - alpha * v_prev
        r = s - omega * t
        x = x + alpha * p_prev + omega * s
        if k > 0:
            xs.append(x.copy())
        if k == iters:
            break
        p = r + beta * (p_prev - omega * v_prev)
        v = G @ p
        # K2
        alpha = rho / np.vdot(rh, v)
        s = r - alpha * v
        t = G @ s
        sums = (np.vdot(t, s), np.vdot(t, t), np.vdot(rh, s), np.vdot(rh, t))
        r_prev, p_prev, v_prev = r, p, v
    return xs


def test_two_pass_iterates_equal_textbook():
    rng = np.random.default_rng(5)
    for n in (12, 40):
        A = rng.normal(size=(n, n))
        G = np.eye(n) * 4.0 + 0.5 * A / np.sqrt(n)        # real, well conditioned, not symmetric
        for _ in range(2):
            b = rng.normal(size=n) + 1j * rng.normal(size=n)
            xa = textbook(G, b, 8)
            xb = two_pass(G, b, 8)
            for a, c in zip(xa, xb):
                assert np.linalg.norm(a - c) <= 1e-10 * np.linalg.norm(a)
            # and the iteration converges to the solution
            xe = np.linalg.solve(G, b)
            assert np.linalg.norm(xb[-1] - xe) < 1e-6 * np.linalg.norm(xe)
