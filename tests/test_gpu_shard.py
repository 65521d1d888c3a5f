"""The sharded state (shard.py) on the GPU, each shard stepped by the
library's kernels through the C ABI (qc_apply_1q, qc_cnot, qc_apply_ctrl,
qc_cphase, Hadamard layers, qc_grover_partial / qc_grover_apply_mean,
qc_norm): world size 1 through the same layer, and 2 or 4 ranks emulated by
host threads of one process on this GPU (the ranks meet only on the host;
no kernel waits on another rank's kernel).  Against the oracle's full-state
result of the same circuit."""
import threading

import numpy as np
import pytest

from shard_cases import circuit, run_oracle, run_sharded

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 2e-5}


@pytest.fixture(scope="module")
def qc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_0902_0699_gb300 as q
    q.lib()
    return q


@pytest.mark.parametrize("dt", [0, 1])
def test_world_size_one_through_the_layer(qc, dt):
    from paper_0902_0699_gb300.shard import LibraryShardOps, ShardedState, TorchComm
    n, seed = 13, 3
    ops = LibraryShardOps(n, dt)
    S = ShardedState(n, ops, TorchComm())
    got = run_sharded(S, circuit(n, seed))
    assert np.max(np.abs(got - run_oracle(n, circuit(n, seed)))) <= TOL[dt]
    assert abs(S.norm2() - 1.0) <= (1e-12 if dt == 0 else 1e-5)
    assert S.exchanges == 0
    ops.close()


@pytest.mark.parametrize("dt", [0, 1])
@pytest.mark.parametrize("world", [2, 4])
def test_thread_ranks_on_one_gpu(qc, dt, world):
    import torch
    from paper_0902_0699_gb300.shard import LibraryShardOps, ShardedState, ThreadComm
    n, seed = 14, 10 + world
    hub = ThreadComm.Hub(world)
    nl = n - (world.bit_length() - 1)
    out, errs = [None] * world, []

    def body(r):
        try:
            torch.cuda.set_device(0)
            ops = LibraryShardOps(nl, dt)
            S = ShardedState(n, ops, ThreadComm(hub, r))
            out[r] = (run_sharded(S, circuit(n, seed)), S.norm2(), S.exchanges)
            torch.cuda.synchronize()
            ops.close()
        except Exception as e:  # reported below
            errs.append(e)
            hub.barrier.abort()

    th = [threading.Thread(target=body, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(600)
    assert not errs, errs
    ref = run_oracle(n, circuit(n, seed))
    for got, nrm, nex in out:
        assert np.max(np.abs(got - ref)) <= TOL[dt]
        assert abs(nrm - 1.0) <= (1e-12 if dt == 0 else 1e-5)
        assert nex > 0
