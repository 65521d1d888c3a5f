"""The sharded state (paper_0902_0699_gb300/shard.py: the paper's
distribution of amplitudes over processes, sec. 3.1-3.3, with the pairwise
exchange for operators on global qubits) on the CPU: gloo ranks in separate
processes (2 and 4) and ranks emulated by threads (8), each shard stepped by
the oracle's gates.  The gathered state must equal the oracle's full-state
result for a circuit that mixes global and local qubits in every gate kind,
with SWAPs as relabellings, Grover steps (one all-reduce each) and the QFT
(exchanges only for Hadamards on global qubits)."""
import os
import socket
import threading

import numpy as np
import pytest
import torch.multiprocessing as mp

from shard_cases import OracleShardOps, circuit, run_oracle, run_sharded


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, seed, q):
    import torch.distributed as dist

    from paper_0902_0699_gb300.shard import ShardedState, TorchComm
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        comm = TorchComm()
        nl = n - (world.bit_length() - 1)
        S = ShardedState(n, OracleShardOps(nl), comm)
        got = run_sharded(S, circuit(n, seed))
        q.put((rank, got, S.norm2(), S.exchanges, list(S.qmap)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_gloo_ranks_match_the_oracle(world):
    n, seed = 8, 40 + world
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, seed, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    ref = run_oracle(n, circuit(n, seed))
    for rank, got, nrm, nex, qmap in res:
        assert np.max(np.abs(got - ref)) <= 1e-12
        assert abs(nrm - 1.0) <= 1e-12
        assert nex > 0  # the global qubits did take the exchange path
        assert sorted(qmap) == list(range(n))


def _thread_ranks(world, n, seed):
    from paper_0902_0699_gb300.shard import ShardedState, ThreadComm
    hub = ThreadComm.Hub(world)
    nl = n - (world.bit_length() - 1)
    out, errs = [None] * world, []

    def body(r):
        try:
            S = ShardedState(n, OracleShardOps(nl), ThreadComm(hub, r))
            out[r] = (run_sharded(S, circuit(n, seed)), S.norm2(), S.exchanges)
        except Exception as e:  # reported below
            errs.append(e)
            hub.barrier.abort()

    th = [threading.Thread(target=body, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(300)
    assert not errs, errs
    return out


def test_thread_ranks_match_the_oracle():
    n, seed = 9, 77
    ref = run_oracle(n, circuit(n, seed))
    for got, nrm, nex in _thread_ranks(8, n, seed):
        assert np.max(np.abs(got - ref)) <= 1e-12
        assert abs(nrm - 1.0) <= 1e-12
        assert nex > 0


def test_single_rank_is_the_plain_state():
    # world size 1: no global qubit, no exchange
    from paper_0902_0699_gb300.shard import ShardedState, TorchComm
    n, seed = 7, 5
    S = ShardedState(n, OracleShardOps(n), TorchComm())
    got = run_sharded(S, circuit(n, seed))
    assert np.max(np.abs(got - run_oracle(n, circuit(n, seed)))) <= 1e-12
    assert S.exchanges == 0


def test_exchange_mapping_by_hand():
    # two thread ranks, n = 3 (one global qubit, bit 2): H on qubit 2 of
    # |1 0 1> (index 5) must move amplitude between the ranks and leave the
    # qubit on the top local bit afterwards
    from paper_0902_0699_gb300.shard import H_MAT, ShardedState, ThreadComm
    hub = ThreadComm.Hub(2)
    res = [None, None]

    def body(r):
        S = ShardedState(3, OracleShardOps(2), ThreadComm(hub, r))
        S.reset(5)
        S.apply_1q(2, H_MAT)
        res[r] = (S.gather(), list(S.qmap), S.exchanges)

    th = [threading.Thread(target=body, args=(r,)) for r in range(2)]
    [t.start() for t in th]
    [t.join(60) for t in th]
    ref = np.zeros(8, dtype=np.complex128)
    ref[1] = 2 ** -0.5
    ref[5] = -(2 ** -0.5)
    for got, qmap, nex in res:
        assert np.allclose(got, ref, atol=1e-15)
        assert qmap == [0, 2, 1] and nex == 1
