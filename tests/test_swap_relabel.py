"""The reading the tiled planner relies on for SWAP runs (CPU only).

A SWAP (three exact CNOTs, Section 1.3 Table 1) only moves amplitudes.  The
planner moves every run of SWAPs to the front of the circuit: with Q the
product of all runs (each run pi, pi[q] = new position of qubit q, applied
in circuit order) and phi = Q, each run met on the way turns phi into
phi o pi^-1 and every other gate acts on phi(its qubits) instead.  Applying Q
to the input first and then the relabelled gates gives the circuit's state,
and phi ends at the identity.  This file restates that transformation on its
own and checks it with the FP64 oracle, so that the property the CUDA path
depends on is pinned independently of it.
"""

import numpy as np
import pytest

from workloads import generators as W


def _swap(a, b):
    X = W.mat_x()
    return [W.gate_record(X, b, (a,)), W.gate_record(X, a, (b,)), W.gate_record(X, b, (a,))]


def _circuit(M, rng, layout):
    """Random gates with SWAP runs where `layout` says ("g" a random gate,
    a tuple of pairs a run of SWAPs).  Returns the records and the runs as
    (first record index, number of SWAPs, permutation)."""
    recs, runs = [], []
    for item in layout:
        if item == "g":
            t = int(rng.integers(M))
            kind = rng.integers(3)
            if kind == 0:
                recs.append(W.gate_record(W.mat_haar_su2(rng), t))
            else:
                c = int(rng.choice([q for q in range(M) if q != t]))
                U = W.mat_haar_su2(rng) if kind == 1 else W.mat_phase(float(rng.uniform(-3, 3)))
                recs.append(W.gate_record(U, t, (c,)))
        else:
            pi = list(range(M))
            start = len(recs)
            for a, b in item:
                recs.extend(_swap(a, b))
                pi = [b if p == a else a if p == b else p for p in pi]
            runs.append((start, len(item), pi))
    return W._pack(recs), runs


def _to_front(recs, runs, M):
    Q = list(range(M))
    for _, _, pi in runs:
        Q = [pi[Q[q]] for q in range(M)]
    phi = Q[:]
    out, i, r = [], 0, 0
    while i < len(recs):
        if r < len(runs) and i == runs[r][0]:
            inv = [0] * M
            for q in range(M):
                inv[runs[r][2][q]] = q
            phi = [phi[inv[q]] for q in range(M)]
            i += 3 * runs[r][1]
            r += 1
            continue
        g = recs[i].copy()
        g["target"] = phi[int(g["target"])]
        for k in range(int(g["ncontrols"])):
            g["controls"][k] = phi[int(g["controls"][k])]
        out.append(g)
        i += 1
    return Q, phi, W._pack(out)


def _permute(x, Q, M):
    """The state after moving the data at qubit position q to Q[q]."""
    idx = np.arange(1 << M)
    y = np.zeros_like(idx)
    for q in range(M):
        y |= ((idx >> q) & 1) << Q[q]
    out = np.empty_like(x)
    out[y] = x
    return out


@pytest.mark.parametrize("layout_id", range(4))
def test_swap_runs_move_to_the_front(orc, layout_id):
    M = 7
    rng = np.random.default_rng(900 + layout_id)
    layouts = [
        ["g"] * 12 + [((0, 6), (1, 5), (2, 4))],                                  # the QFT's closing reversal
        ["g"] * 6 + [((0, 3),)] + ["g"] * 6 + [((1, 5), (2, 6))] + ["g"] * 4,      # runs in the middle
        [((0, 1), (1, 2))] + ["g"] * 10,                                          # a 3-cycle at the start
        ["g"] * 5 + [((4, 5),)] + ["g"] * 5 + [((4, 5),)] + ["g"] * 5,           # a run and its inverse
    ]
    recs, runs = _circuit(M, rng, layouts[layout_id])
    x = W.random_state(M, seed=3, dtype=np.complex128)
    ref = orc.run(M, recs, x)
    Q, phi, rel = _to_front(recs, runs, M)
    assert phi == list(range(M))
    got = orc.run(M, rel, _permute(x, Q, M))
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
    assert len(rel) == len(recs) - 3 * sum(n for _, n, _ in runs)
