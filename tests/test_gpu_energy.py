"""Direct parity of the element pass, the barrier pass and the assembly (rows
a2-a5): the incremental potential and its gradient evaluated by the GPU at
positions and an indenter pose taken from the oracle's converged contact
state equal the oracle's (brute-force candidate pairs) -- a GPU candidate set
missing any pair closer than dhat would lower the energy.  The states are
1e-3 dhat off equilibrium, where the assembled gradient is still a near
cancellation of elastic and barrier forces: in the FP32 mode it carries
~1e-3 relative rounding (FP64: 1e-9)."""
import numpy as np
import pytest

from gpu_util import rel_fro
from oracle.sim import Scene
from synth import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,etol,gtol", [("fp64", 1e-10, 1e-9), ("fp32", 1e-5, 2e-3)])
@pytest.mark.parametrize("seed", [0, 5])
def test_energy_gradient_in_contact(precision, etol, gtol, seed):
    from paper_2606_20426_gb300 import Env
    env = workloads.small_env(seed)
    ref = Scene(env)
    ref.step(env["poses"][0])
    # off equilibrium (a converged gradient is a cancellation of elastic and
    # barrier forces): displace the free vertices by ~1e-3 dhat, far less than
    # the gaps the barrier keeps
    rng = np.random.default_rng(seed)
    x = ref.x + 1e-3 * env["opts"]["dhat"] * rng.standard_normal(ref.x.shape) * ref.free[:, None]
    Y = ref.indenter(env["poses"][0])
    cand = ref.candidates(x, Y)
    Eref = ref.energy(x, Y, cand)
    _, gref, _ = ref.gradient_hessian(x, Y)
    gref = gref.reshape(-1, 3)
    gref[~ref.free] = 0.0
    g = Env(env, precision=precision)
    g.step(env["poses"][0])  # the GPU env now sits at the same indenter pose
    g.set_positions(x)
    E, grad = g.energy_gradient()
    g.close()
    assert abs(E - Eref) <= etol * abs(Eref)
    assert rel_fro(grad, gref) <= gtol
    # the state is in contact: the barrier term is active
    Eb, _ = ref.barrier_terms(x, Y, cand, need_hess=False)
    assert Eb > 0.0
