"""The force/torque error metric of the parity tests: each body's wrench
(F, T / R), normalised by the oracle's maximum of that series; a body whose
wrench vanishes in the oracle (zero by symmetry) is measured against its
characteristic force rho0 U^2 R^(D-1)."""
import numpy as np

from parity_util import VANISHING, char_scales, ft_rel_error, ft_series_errors

SPEC = dict(lattice="D2Q9", n=(64, 32), tau=0.7,
            bodies=[dict(shape="cylinder", R=10.0, X0=(20.0, 16.0), U=(0.02, 0.0)),
                    dict(shape="cylinder", R=5.0, X0=(50.0, 16.0))])


def test_wrench_normalisation():
    fc, tc = char_scales(SPEC)[0]
    assert np.isclose(fc, 0.02 ** 2 * 10.0) and np.isclose(tc, fc * 10.0)
    steps = 7
    ref = np.zeros((steps, 2, 6))
    ref[:, 0, 0] = np.linspace(0.1, 1.0, steps) * 3e-2  # drag of body 0, max 3e-2
    ref[:, 0, 5] = 1e-5  # a torque far below R |F| = 0.3
    ref[:, 1, 1] = 1e-17 * np.arange(steps)  # body 1: round-off of a zero wrench
    got = ref.copy()
    got[3, 0, 5] += 6e-7  # torque error: 6e-7 / R = 6e-8 against the wrench max 3e-2
    assert np.isclose(ft_rel_error(got, ref, SPEC), 6e-8 / 3e-2)
    assert ft_series_errors(got, ref)[0][1] > 5e-2  # against its own tiny maximum
    got = ref.copy()
    got[2, 0, 1] += 3e-6  # lift error against the drag maximum
    assert np.isclose(ft_rel_error(got, ref, SPEC), 1e-4)
    got = ref.copy()
    got[4, 1, 0] += 2e-9  # body 1 vanishes: measured against its F_c
    fc1 = char_scales(SPEC)[1][0]
    assert np.isclose(ft_rel_error(got, ref, SPEC), 2e-9 / fc1)
    assert VANISHING < 1e-6
    # the subset form used for sampled bodies
    assert np.isclose(ft_rel_error(got[:, 1:2], ref[:, 1:2], SPEC, bodies=[1]), 2e-9 / fc1)
    # without a problem description: force and torque each against their own maximum
    got = ref.copy()
    got[3, 0, 0] += 3e-6
    assert np.isclose(ft_rel_error(got[:, :1], ref[:, :1]), 1e-4)
