"""The GPU twin of the Metropolis gauge-field generator (inputs/metropolis_gpu.cu) runs the
CPU generator's Markov chain: same angles bit for bit, same acceptance, and the stored
digests of the CPU-made workload fields. Fields at sizes the CPU generator cannot make
inside a test or a bench (1024^2, the many-field ensembles) come from this twin, and
their digests are checked the same way where a stored digest exists."""
import numpy as np
import pytest

import inputs
from tests._util import mcrit_table

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L0,L1,beta,sweeps", [(64, 64, 6.0, 2000), (32, 48, 3.0, 300), (16, 8, 10.0, 500)])
def test_gpu_chain_equals_cpu_chain(L0, L1, beta, sweeps):
    seed = inputs.member_seed(7, L0, beta, 3)
    th_cpu, acc_cpu = inputs.metropolis_u1_2d(L0, L1, beta, sweeps, seed)
    th_gpu, acc_gpu = inputs.metropolis_u1_2d_gpu(L0, L1, [beta], [seed], sweeps)
    assert np.array_equal(th_gpu[0], th_cpu)
    assert acc_gpu[0] == acc_cpu


def test_gpu_batch_of_fields_equals_cpu_fields():
    L, sweeps = 32, 400
    betas = [3.0, 6.0, 10.0, 6.0]
    seeds = [inputs.member_seed(8, L, b, i) for i, b in enumerate(betas)]
    th, acc = inputs.metropolis_u1_2d_gpu(L, L, betas, seeds, sweeps)
    for k in range(len(seeds)):
        ref, a = inputs.metropolis_u1_2d(L, L, betas[k], sweeps, seeds[k])
        assert np.array_equal(th[k], ref) and acc[k] == a


@pytest.mark.parametrize("key", ["w1_L256_b6", "w1_L256_b10"])
def test_gpu_chain_reproduces_stored_workload_digests(key):
    row = mcrit_table()[key]
    th, acc = inputs.metropolis_u1_2d_gpu(row["L"], row["L"], [row["beta"]], [row["seed"]], row["sweeps"])
    assert inputs.field_digest(th[0]) == row["theta_digest"]
    assert abs(acc[0] - row["acceptance"]) < 1e-15
