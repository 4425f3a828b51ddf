"""The patch cut on the CPU: the oracle on a patch reproduces the oracle on
the whole mesh at the seed elements, for the operator, one ADER step and
one LSRK step (the domains of dependence the full-size GPU tests rely on)."""
import numpy as np

import oracle
import synth
from patch_helpers import patch


def _cfg():
    rng = np.random.default_rng(7)
    mesh = synth.cube_mesh(6, q=2, periodic=True, deform=synth.mesh.curving(0.05),
                           frames=synth.mesh.random_frames(216, rng))
    x = synth.solution_node_positions(mesh, 2)
    rho, c = synth.fields.cfg2_coefficients(x)
    return mesh, rho, c, synth.configs.random_state(216, 2, 8)


def test_patch_reproduces_whole_mesh():
    mesh, rho, c, U = _cfg()
    whole = oracle.Oracle(mesh, 2, rho, c, 1.0)
    seeds = [0, 77, 215]
    for radius, run in ((1, lambda o, V: o.apply(V)), (1, lambda o, V: o.ader(V, 0.01, 1, 2)),
                        (5, lambda o, V: o.lsrk(V, 0.01, 1))):
        ref = run(whole, U)[seeds]
        sub, ids, r, cc, V, loc = patch(mesh, rho, c, U, seeds, radius)
        assert sub["n_elem"] < 216 or radius == 5
        got = run(oracle.Oracle(sub, 2, r, cc, 1.0), V)[loc]
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref)), radius
    # one layer short, the seeds see the cut (the test above is not vacuous)
    sub, ids, r, cc, V, loc = patch(mesh, rho, c, U, seeds, 0)
    got = oracle.Oracle(sub, 2, r, cc, 1.0).apply(V)[loc]
    assert np.max(np.abs(got - whole.apply(U)[seeds])) > 1e-3
