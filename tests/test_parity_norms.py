"""The parity gates used by the GPU tests, checked on the CPU with a mistake
planted in an oracle result: one point value off by 1% on a 37 x 29 grid
stays under the whole-array relative L1 gate of 1e-5 but fails the
per-element gate, which names its place."""
import numpy as np
import pytest

from helpers import make_oracle
from test_gpu_parity import STEP_TOL, _flow, assert_parity, state_err, state_max_err


def _one_step(oracle_mod):
    prob = _flow((1.0, -0.5, 0.4, 1.0))
    o = make_oracle(oracle_mod, prob)
    o.step(0.3 * prob.dx / o.max_speed())
    return [np.array(a) for a in o.get_state()]


def test_identical_states_pass_both_gates(oracle_mod):
    want = _one_step(oracle_mod)
    l1, e = assert_parity([a.copy() for a in want], want, STEP_TOL)
    assert l1 == 0.0 and e == 0.0


@pytest.mark.parametrize("array,var", [(1, 0), (2, 1), (3, 3), (0, 2)])
def test_one_wrong_value_fails_only_the_element_gate(oracle_mod, array, var):
    want = _one_step(oracle_mod)
    got = [a.copy() for a in want]
    j, i = 7, 11
    got[array][var, j, i] += 0.01 * max(abs(want[array][var, j, i]), 0.5)
    assert state_err(got, want) < STEP_TOL  # the L1 gate alone misses it
    e, k, v, idx, _, _ = state_max_err(got, want)
    assert (k, v, idx) == (array, var, (j, i)) and e > 1e-3
    with pytest.raises(AssertionError, match=f"array {array} variable {var} index \\({j}, {i}\\)"):
        assert_parity(got, want, STEP_TOL)
