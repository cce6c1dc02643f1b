"""Failure detection on the GPU without a fault: the fused tensor-core
kernel bounds every pipeline wait.  With the bound set to 1 microsecond
(qsim_opts.wait_us) its waits run out, the kernel records QSIM_ETIMEOUT,
drains its copies and MMAs in flight (those waits keep the full 2 s bound),
frees its tensor memory and returns; qsim_plan_status reports the timeout
once, and the device stays usable: the same circuit with the default bound
then matches the oracle."""

import os

import numpy as np
import pytest

import paper_quant_ph_9804039_gb300 as qs
from workloads import generators as W

pytestmark = pytest.mark.gpu

NT = max(1, os.cpu_count() or 1)


def _gates(rng, qubits, n):
    recs = []
    for _ in range(n):
        t = int(rng.choice(qubits))
        recs.append(W.gate_record(W.mat_haar_su2(rng), t))
    return W._pack(recs)


@pytest.mark.parametrize("qubits", [(0, 1, 2, 3, 4), (12, 13, 14, 15, 16)])
def test_fused_wait_timeout_is_reported_and_recovered(orc, qubits):
    M = 20
    rng = np.random.default_rng(sum(qubits))
    recs = _gates(rng, list(qubits), 30)
    x = W.random_state(M, seed=2)
    short = qs.Plan(M, recs, mode="fused", fuse_k=5, wait_us=1)
    assert short.stats()["mode"] == qs.MODE_FUSED
    st = qs.State(M).set(x)
    short.execute(st)
    with pytest.raises(qs.QsimError) as e:
        short.status()
    assert e.value.code == qs.QSIM_ETIMEOUT
    short.status()  # the record was cleared
    good = qs.Plan(M, recs, mode="fused", fuse_k=5)
    st2 = qs.State(M).set(x)
    good.execute(st2)
    good.status()
    ref = orc.run(M, recs, x.astype(np.complex128), nthreads=NT)
    got = st2.get().astype(np.complex128)
    assert np.abs(got - ref).max() <= 1e-5 and np.linalg.norm(got - ref) <= 1e-5
