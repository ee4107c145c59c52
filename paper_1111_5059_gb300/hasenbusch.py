"""Hasenbusch mass ladders (Sec. 3): construction and continuous tuning.

The determinant ratio of the light quark over its Pauli-Villars partner is
split into k + 1 quotient terms with intermediate masses

    det(D+(m)D(m) / D+(1)D(1)) = prod_{i=1}^{k+1} det(D+(m_{i-1})D(m_{i-1}) / D+(m_i)D(m_i)),
    m = m_0 < m_1 < ... < m_{k+1} = 1,

(the paper writes m_i = m + mu_i; the product telescopes to the left-hand side
only with the last mass equal to the Pauli-Villars mass 1, so m_{k+1} = 1).
The intermediate masses are free continuous parameters.  The paper tunes them
so that no term carries a large force, which lets every force-term Dirac
equation be solved to 1e-6 instead of 1e-8; here "tuned" means the terms'
force norms are equal.

This module is host logic only: it chooses masses and drives a caller-supplied
function that measures the terms' force norms (on the GPU in the benchmark),
and holds none of the method's arithmetic.
"""
from __future__ import annotations

import math
from typing import Callable, List, Sequence, Tuple


def geometric_ladder(m: float, k: int, m_pv: float = 1.0) -> List[float]:
    """m_0 = m, ..., m_{k+1} = m_pv with equal ratios m_{i+1} / m_i."""
    if not (0.0 < m < m_pv) or k < 0:
        raise ValueError("need 0 < m < m_pv and k >= 0")
    r = (m_pv / m) ** (1.0 / (k + 1))
    masses = [m * r ** i for i in range(k + 2)]
    masses[-1] = m_pv
    return masses


def terms(masses: Sequence[float]) -> List[Tuple[float, float]]:
    """The quotient terms (m_{i-1}, m_i) of a ladder."""
    if any(b <= a for a, b in zip(masses, masses[1:])):
        raise ValueError("ladder masses must increase")
    return [(a, b) for a, b in zip(masses, masses[1:])]


def tune_ladder(masses: Sequence[float], force_norms: Callable[[List[Tuple[float, float]]], Sequence[float]],
                iters: int = 8, rtol: float = 0.05, gamma: float = 1.0):
    """Move the intermediate masses until the terms' force norms are equal.

    In log-mass coordinates term i spans a width w_i = log(m_i / m_{i-1}); the
    end points stay fixed.  Each step measures the norms F_i and rescales
    w_i <- w_i (F_bar / F_i)^gamma, F_bar their geometric mean, keeping the sum
    of the widths: a term whose force is above the others gets a narrower
    mass ratio.  For forces that grow like a power of the width this is a
    Newton-like step.  Stops when max F / min F - 1 < rtol.

    Returns (masses, history) with history a list of (masses, norms).
    """
    ms = list(masses)
    terms(ms)  # validates
    if len(ms) < 3:
        return ms, [(ms, list(force_norms(terms(ms))))]
    x = [math.log(v) for v in ms]
    total = x[-1] - x[0]
    history = []
    for _ in range(iters):
        f = [float(v) for v in force_norms(terms(ms))]
        history.append((list(ms), f))
        if min(f) <= 0.0:
            raise ValueError("force norms must be positive")
        if max(f) / min(f) - 1.0 < rtol:
            break
        w = [b - a for a, b in zip(x, x[1:])]
        fbar = math.exp(sum(math.log(v) for v in f) / len(f))
        w = [wi * (fbar / fi) ** gamma for wi, fi in zip(w, f)]
        s = sum(w)
        w = [wi * total / s for wi in w]
        x = [x[0]]
        for wi in w[:-1]:
            x.append(x[-1] + wi)
        x.append(math.log(ms[-1]))
        ms = [ms[0]] + [math.exp(v) for v in x[1:-1]] + [ms[-1]]
    else:
        history.append((list(ms), [float(v) for v in force_norms(terms(ms))]))
    return ms, history
