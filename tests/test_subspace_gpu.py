"""Touched-qubit subspace (qsim_opts.subspace; Section 3.2, Figure 7, EQ 6):
a circuit applied to |0...0> runs each gate only on the prefix of the vector
that the qubits touched so far span, then restores the qubit order.  Against
the oracle (from |0...0>) and the flat plan, in every execution form, with
touch orders that need no relabelling, one involution, or two."""

import os

import numpy as np
import pytest

import paper_quant_ph_9804039_gb300 as qs
from workloads import generators as W

pytestmark = pytest.mark.gpu

NT = max(1, os.cpu_count() or 1)


def _close(got, ref):
    d = np.abs(got.astype(np.complex128) - ref)
    assert d.max() <= 1e-5, d.max()
    assert np.linalg.norm(got.astype(np.complex128) - ref) <= 1e-5


def _orders(M):
    rng = np.random.default_rng(M)
    return {"ascending": list(range(M)), "descending": list(range(M - 1, -1, -1)),
            "random": [int(v) for v in rng.permutation(M)]}


@pytest.mark.parametrize("order", ["ascending", "descending", "random"])
@pytest.mark.parametrize("mode", ["tiled", "fused", "unfused"])
def test_gradual_circuit_against_oracle(orc, order, mode):
    M = 20
    c = W.circuit_gradual(M, start=3, per_qubit=12, order=_orders(M)[order])
    sub = qs.Plan(M, c["noisy"], mode=mode, subspace=True)
    desc = sub.describe()
    assert "subspace:" in desc
    nseg = int(desc.split("subspace: ")[1].split()[0])
    assert nseg >= 2, desc[:400]
    st = qs.State(M)
    st.set(W.random_state(M, seed=9))  # overwritten: the plan starts from |0...0>
    sub.execute(st)
    sub.status()
    ref = orc.run(M, c["noisy"], nthreads=NT)
    got = st.get()
    _close(got, ref)
    flat = qs.State(M)
    qs.Plan(M, c["noisy"], mode=mode).execute(flat)
    _close(flat.get(), ref)


@pytest.mark.parametrize("mode", ["tiled", "fused"])
def test_gradual_fidelity(orc, mode):
    """Ideal and noisy subspace plans: F and the norm as the oracle's."""
    M = 22
    c = W.circuit_gradual(M, start=4, per_qubit=10, order=_orders(M)["random"])
    a, b = qs.State(M), qs.State(M)
    qs.Plan(M, c["ideal"], mode=mode, subspace=True).execute(a)
    qs.Plan(M, c["noisy"], mode=mode, subspace=True).execute(b)
    F, nrm = qs.fidelity(a, b)
    Fo, nrmo = orc.fidelity(orc.run(M, c["ideal"], nthreads=NT), orc.run(M, c["noisy"], nthreads=NT))
    assert abs(F - Fo) <= 1e-6 and abs(nrm - nrmo) <= 1e-6
    assert F < 1.0 - 1e-6


def test_untouched_controls_and_phases(orc):
    """Gates controlled by untouched qubits are left out; diagonal gates on
    untouched targets (before anything is touched, and after) become factors;
    a circuit of such gates alone leaves a multiple of |0...0>."""
    M = 12
    rz = W.mat_rz(0.7)
    recs = [W.gate_record(rz, 5), W.gate_record(W.mat_x(), 3, (7,)), W.gate_record(np.diag([1j, -1.0]), 2),
            W.gate_record(W.mat_haar_su2(np.random.default_rng(1)), 4), W.gate_record(rz, 9, (4,)),
            W.gate_record(W.mat_phase(0.3), 1, (4,)), W.gate_record(W.mat_x(), 6, (4, 8))]
    recs = W._pack(recs)
    plan = qs.Plan(M, recs, mode="tiled", subspace=True)
    desc = plan.describe()
    assert "3 gates left out" in desc, desc[:300]  # CNOT(7->3), Toffoli(4,8->6), and the phase with U00 = 1
    st = qs.State(M)
    plan.execute(st)
    _close(st.get(), orc.run(M, recs))
    only = W._pack([W.gate_record(rz, 5), W.gate_record(np.diag([1j, -1.0]), 2)])
    st2 = qs.State(M)
    qs.Plan(M, only, mode="tiled", subspace=True).execute(st2)
    _close(st2.get(), orc.run(M, only))
    empty = qs.State(M)
    empty.set(W.random_state(M, seed=3))
    qs.Plan(M, only[:0], mode="tiled", subspace=True).execute(empty)
    assert np.array_equal(empty.get(), orc.zero_state(M).astype(np.complex64))


def test_subspace_saves_work():
    """The planned amplitude updates of the gradual circuit are a fraction of
    the flat count (EQ 6 against EQ 5)."""
    M = 24
    c = W.circuit_gradual(M, start=4, per_qubit=16)
    desc = qs.Plan(M, c["noisy"], mode="tiled", subspace=True).describe()
    line = desc.split("subspace: ")[1].splitlines()[0]
    done = float(line.split("amp-updates ")[1].split()[0])
    flat = float(line.split(" of ")[1].split()[0])
    assert done < 0.25 * flat, line
