"""The oracle against what the paper and the mathematics fix (CPU only)."""

import numpy as np
import pytest

from oracle_pins import PINS
from workloads import generators as W


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(orc, pin):
    pin(orc)


def test_threads_split_is_exact(orc):
    """Splitting the index range over host threads changes no bit."""
    c = W.circuit_c1_random(M=14, n_gates=40)
    x = W.random_state(14, seed=2, dtype=np.complex128)
    a = orc.run(14, c["noisy"], x, nthreads=1)
    b = orc.run(14, c["noisy"], x, nthreads=4)
    assert np.array_equal(a, b)


def test_rejects_bad_gates(orc):
    psi = orc.zero_state(3)
    for t, ctl in ((3, ()), (-1, ()), (0, (0,)), (0, (1, 1)), (0, (5,))):
        with pytest.raises(ValueError):
            orc.apply_gate(psi, W.mat_x(), t, ctl)
