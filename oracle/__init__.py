"""FP64 CPU oracle for the phylogenetic log-likelihood and its gradient.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it. It shares
no code, tables or constants with the CUDA library; the two meet only in the
seeded inputs of ``synth``.

Contents (each function cites the passage it follows):

* ``model``     -- rate matrices Q for HKY85, GTR and GY94 (F3x4), normalised
                   to one expected substitution per unit time, and dQ/dtheta.
* ``pruning``   -- transition matrices by ``scipy.linalg.expm``, Felsenstein
                   post-order pruning with optional power-of-two rescaling,
                   root log-likelihood (Sec. "Algorithmic advances").
* ``gradient``  -- pre-order partials, branch-length gradient by the
                   pre-order . dP/dt . post-order sandwich (Sec. "Algorithmic
                   advances", Sec. "Discussion"), substitution-parameter
                   gradient through the Frechet derivative of expm.
* ``brute``     -- the likelihood by its definition: a sum over every
                   assignment of states to internal nodes (tiny trees only).

Every function is pinned by ``tests/test_oracle.py`` to closed forms,
brute force, invariants or finite differences; none is "parity unpinned".
"""
from . import model, pruning, gradient, brute  # noqa: F401
