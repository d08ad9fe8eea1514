"""Substitution-model rate matrices (oracle; test infrastructure only).

The paper benchmarks HKY85 and GY94 (Sec. "Scaling by number of taxa and
site patterns") and GTR (Sec. "ARM NEON"); the CTMC rate matrix Q is the
object whose eigendecomposition gives the transition matrices (Sec.
"Discussion"). Readings where the paper is silent:

* states are A,C,G,T for nucleotides and the 61 sense codons of the standard
  genetic code in ACGT-lexicographic order (stops TAA, TAG, TGA removed);
* Q_ij = s_ij * pi_j for i != j, Q_ii = -sum_j Q_ij, then Q <- Q / mu with
  mu = -sum_i pi_i Q_ii (one expected substitution per unit time, per site
  for nucleotides and per codon for GY94);
* dQ/dtheta differentiates the normalised matrix, normaliser included.
"""
from __future__ import annotations

import numpy as np

BASES = "ACGT"
# Standard genetic code (NCBI table 1), first/second/third base in T,C,A,G
# order, '*' = stop.
_CODE_TCAG = "FFLLSSSSYY**CC*WLLLLPPPPHHQQRRRRIIIMTTTTNNKKSSRRVVVVAAAADDEEGGGG"


def genetic_code():
    """Return (codons, amino) for the 61 sense codons in ACGT order; each codon
    is a tuple of base indices into BASES."""
    tcag = "TCAG"
    aa_of = {}
    k = 0
    for a in tcag:
        for b in tcag:
            for c in tcag:
                aa_of[(BASES.index(a), BASES.index(b), BASES.index(c))] = _CODE_TCAG[k]
                k += 1
    codons, amino = [], []
    for a in range(4):
        for b in range(4):
            for c in range(4):
                if aa_of[(a, b, c)] != "*":
                    codons.append((a, b, c))
                    amino.append(aa_of[(a, b, c)])
    return codons, amino


def _is_transition(x: int, y: int) -> bool:
    """A<->G and C<->T are transitions; the other changes are transversions."""
    return {x, y} in ({0, 2}, {1, 3})


def _normalise(R: np.ndarray, pi: np.ndarray, dR: list[np.ndarray]):
    """Fill the diagonal, divide by mu = -sum_i pi_i Q_ii, and differentiate."""
    R = R.copy()
    np.fill_diagonal(R, 0.0)
    np.fill_diagonal(R, -R.sum(axis=1))
    mu = -np.dot(pi, np.diag(R))
    Q = R / mu
    dQ = []
    for D in dR:
        D = D.copy()
        np.fill_diagonal(D, 0.0)
        np.fill_diagonal(D, -D.sum(axis=1))
        dmu = -np.dot(pi, np.diag(D))
        dQ.append(D / mu - R * dmu / mu**2)
    return Q, dQ


def hky(kappa: float, pi) -> tuple[np.ndarray, list[np.ndarray]]:
    """HKY85: s_ij = kappa for transitions, 1 for transversions.
    Returns (Q, [dQ/dkappa])."""
    pi = np.asarray(pi, float)
    R = np.zeros((4, 4), dtype=np.result_type(kappa, float))
    D = np.zeros((4, 4))
    for i in range(4):
        for j in range(4):
            if i != j:
                ts = _is_transition(i, j)
                R[i, j] = (kappa if ts else 1.0) * pi[j]
                D[i, j] = (1.0 if ts else 0.0) * pi[j]
    return _normalise(R, pi, [D])


GTR_PAIRS = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))  # AC AG AT CG CT GT


def gtr(rates, pi) -> tuple[np.ndarray, list[np.ndarray]]:
    """GTR: symmetric exchangeabilities s_ij in the order AC, AG, AT, CG, CT, GT.
    Returns (Q, [dQ/drate_k for k in 0..5])."""
    pi = np.asarray(pi, float)
    rates = np.asarray(rates)
    rates = rates.astype(np.result_type(rates.dtype, float))
    R = np.zeros((4, 4), dtype=rates.dtype)
    dR = [np.zeros((4, 4)) for _ in range(6)]
    for k, (i, j) in enumerate(GTR_PAIRS):
        R[i, j] = rates[k] * pi[j]
        R[j, i] = rates[k] * pi[i]
        dR[k][i, j] = pi[j]
        dR[k][j, i] = pi[i]
    return _normalise(R, pi, dR)


def f3x4_frequencies(f3x4) -> np.ndarray:
    """F3x4 codon frequencies: pi_c proportional to f1[c1] f2[c2] f3[c3] over
    the 61 sense codons (renormalised after removing the stops)."""
    f = np.asarray(f3x4, float)
    codons, _ = genetic_code()
    pi = np.array([f[0, a] * f[1, b] * f[2, c] for (a, b, c) in codons])
    return pi / pi.sum()


def gy94_pairs() -> list[tuple[int, int]]:
    """Unordered pairs (i < j, lexicographic) of sense codons that differ at
    exactly one position: the non-zero off-diagonal elements of GY94 (263)."""
    codons, _ = genetic_code()
    return [(i, j) for i in range(len(codons)) for j in range(i + 1, len(codons))
            if sum(codons[i][k] != codons[j][k] for k in range(3)) == 1]


def gy94(kappa, omega, f3x4, eps=None):
    """Goldman-Yang 1994 codon model on the 61 sense codons.

    s_ij = 0 unless codons i and j differ at exactly one position; otherwise
    s_ij = kappa^[transition] * omega^[nonsynonymous]. pi is F3x4.
    ``eps`` (one value per pair of gy94_pairs()) adds random effects: s_ij
    and s_ji are multiplied by exp(eps_k) (Sec. "Algorithmic advances":
    multiplicative random effects on the non-diagonal elements; symmetric
    here, so Q stays reversible). Any argument may be complex (complex-step
    derivatives). Returns (Q, pi, [dQ/dkappa, dQ/domega])."""
    codons, amino = genetic_code()
    pi = f3x4_frequencies(f3x4)
    n = len(codons)
    dt = np.result_type(kappa, omega, float if eps is None else np.asarray(eps).dtype)
    mult = np.ones((n, n), dtype=dt)
    if eps is not None:
        for k, (i, j) in enumerate(gy94_pairs()):
            mult[i, j] = mult[j, i] = np.exp(eps[k])
    R = np.zeros((n, n), dtype=dt)
    Dk = np.zeros((n, n), dtype=dt)
    Dw = np.zeros((n, n), dtype=dt)
    for i, ci in enumerate(codons):
        for j, cj in enumerate(codons):
            diff = [k for k in range(3) if ci[k] != cj[k]]
            if len(diff) != 1:
                continue
            pos = diff[0]
            ts = _is_transition(ci[pos], cj[pos])
            ns = amino[i] != amino[j]
            k_ = kappa if ts else 1.0
            w_ = omega if ns else 1.0
            R[i, j] = k_ * w_ * pi[j] * mult[i, j]
            Dk[i, j] = (1.0 if ts else 0.0) * w_ * pi[j] * mult[i, j]
            Dw[i, j] = k_ * (1.0 if ns else 0.0) * pi[j] * mult[i, j]
    Q, dQ = _normalise(R, pi, [Dk, Dw])
    return Q, pi, dQ


def rev(exch, pi):
    """General reversible model on len(pi) states: s_ij = (E_ij + E_ji) / 2 for
    the S x S exchangeability matrix E (diagonal ignored). Returns Q."""
    pi = np.asarray(pi, float)
    S = len(pi)
    E = np.asarray(exch).reshape(S, S)
    E = 0.5 * (E + E.T)
    R = E * pi[None, :]
    return _normalise(R, pi, [])[0]


def build(model: str, params, freqs):
    """(Q, pi, [dQ/dtheta]) for model in {"hky", "gtr", "gy94", "gy94re", "rev"}
    ("gy94re": params kappa, omega, then one random effect per pair of
    gy94_pairs(); the dQ list covers kappa and omega; "rev": params the S x S
    exchangeabilities, no dQ list)."""
    if model == "hky":
        Q, dQ = hky(params[0], freqs)
        return Q, np.asarray(freqs, float), dQ
    if model == "gtr":
        Q, dQ = gtr(params, freqs)
        return Q, np.asarray(freqs, float), dQ
    if model == "gy94":
        return gy94(params[0], params[1], freqs)
    if model == "gy94re":
        return gy94(params[0], params[1], freqs, np.asarray(params[2:]))
    if model == "rev":
        return rev(params, freqs), np.asarray(freqs, float), []
    raise ValueError(model)


def rate_jacobian(model: str, params, freqs, h: float = 1e-30) -> np.ndarray:
    """dQ/dtheta_k for every parameter k ([K, S, S]) by complex-step
    differentiation of the builder: Im Q(theta + i h e_k) / h, exact to
    rounding (no subtraction), independent of the hand-written dQ."""
    params = np.asarray(params, float).ravel()
    out = []
    for k in range(len(params)):
        z = params.astype(complex)
        z[k] += 1j * h
        out.append(build(model, z, freqs)[0].imag / h)
    return np.array(out)
