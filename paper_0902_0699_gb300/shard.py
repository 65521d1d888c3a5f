"""A state vector split over several devices (one shard per rank).

The QCMPI paper spreads the 2^n amplitudes over MPI processes (sec. 3.1-3.3)
and pairs every amplitude with its partner by a SEND/RECV exchange when an
operator acts on a qubit whose partner lives on another process.  Here the
same idea is recast for GPUs:

* World size P = 2^p; rank r holds the 2^(n-p) amplitudes whose p highest
  physical index bits equal r (a contiguous slice), so bits [0, n-p) are
  local and bits [n-p, n) select the rank.
* A logical -> physical qubit map is kept.  SWAP is a relabelling (no data
  moves), and so is the QFT's final bit reversal.
* A one-qubit or controlled operator whose target sits on a global bit g
  first swaps g with the top local bit L = n-p-1: rank r and its partner
  r ^ 2^(g-(n-p)) exchange the half of their shard whose bit L differs from
  their own bit g (one contiguous half, S/2 bytes each way) -- the paper's
  pairwise exchange -- after which the target is local.  Controls on global
  bits need no exchange (the rank either applies the operator or not), and
  diagonal operators (CPHASEK, the oracle) never do.
* The Grover diffusion 2|s><s| - I does not depend on the qubit order: each
  rank sends one complex partial sum (an all-reduce), then runs the
  single-device fused pass with the global mean.
* Norms are one scalar all-reduce.

Every operation on a shard runs through a `ShardOps` object (the library's
kernels on the shard, via `LibraryShardOps`); exchanges and reductions go
through a `Comm` (torch.distributed with NCCL or gloo, via `TorchComm`, or
ranks emulated by threads of one process, via `ThreadComm`).
"""
from __future__ import annotations

import math
import threading

import numpy as np

H_MAT = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)
X_MAT = np.array([[0, 1], [1, 0]], dtype=np.complex128)


# ----------------------------------------------------------- communicators --

class TorchComm:
    """Exchanges and reductions over torch.distributed (NCCL for CUDA
    tensors, gloo for CPU tensors)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1

    def _peer(self, r):
        return r if self.group is None else self.dist.get_global_rank(self.group, r)

    def sendrecv(self, send, recv, partner):
        import torch
        a, b = torch.view_as_real(send), torch.view_as_real(recv)
        ops = [self.dist.P2POp(self.dist.isend, a, self._peer(partner), self.group),
               self.dist.P2POp(self.dist.irecv, b, self._peer(partner), self.group)]
        for req in self.dist.batch_isend_irecv(ops):
            req.wait()

    def allreduce(self, values, device):
        import torch
        t = torch.tensor(np.asarray(values, dtype=np.float64), device=device)
        if self.world > 1:
            self.dist.all_reduce(t, group=self.group)
        return t.cpu().numpy()

    def allgather(self, tensor):
        import torch
        if self.world == 1:
            return [tensor.clone()]
        parts = [torch.empty_like(torch.view_as_real(tensor)) for _ in range(self.world)]
        self.dist.all_gather(parts, torch.view_as_real(tensor).contiguous(), group=self.group)
        return [torch.view_as_complex(p) for p in parts]


class ThreadComm:
    """Ranks emulated by the threads of one process (one per rank): host-side
    rendezvous and copies, so no device work ever waits on another rank's
    device work.  `Hub` is shared by the ranks; each rank gets its own
    ThreadComm(hub, rank)."""

    class Hub:
        def __init__(self, world):
            self.world = world
            self.barrier = threading.Barrier(world)
            self.slots = [None] * world

    def __init__(self, hub, rank):
        self.hub, self.rank, self.world = hub, rank, hub.world

    def _sync_device(self, tensor):
        if tensor.is_cuda:
            import torch
            torch.cuda.current_stream(tensor.device).synchronize()

    def sendrecv(self, send, recv, partner):
        self._sync_device(send)
        self.hub.slots[self.rank] = send
        self.hub.barrier.wait()  # every rank's data is ready
        recv.copy_(self.hub.slots[partner])
        self._sync_device(recv)
        self.hub.barrier.wait()  # every copy is done before anyone overwrites `send`
        self.hub.slots[self.rank] = None

    def allreduce(self, values, device):
        self.hub.slots[self.rank] = np.asarray(values, dtype=np.float64)
        self.hub.barrier.wait()
        out = np.sum(np.stack(self.hub.slots), axis=0)
        self.hub.barrier.wait()
        return out

    def allgather(self, tensor):
        self._sync_device(tensor)
        self.hub.slots[self.rank] = tensor
        self.hub.barrier.wait()
        parts = [t.clone() for t in self.hub.slots]
        self.hub.barrier.wait()
        return parts


# ------------------------------------------------------------ shard operations --

class LibraryShardOps:
    """The library's kernels on one shard (a state of n - p qubits on this
    rank's GPU)."""

    def __init__(self, nl: int, dt: int, stream=None):
        from . import State
        self.state = State(nl, dt, stream=stream)
        self.tensor = self.state.tensor
        self.device = self.tensor.device

    def zero(self, local_index=None):
        if local_index is None:
            self.tensor.zero_()
            from . import qc_state_invalidate
            qc_state_invalidate(self.state.h)
        else:
            self.state.reset(int(local_index))

    def invalidate(self):
        from . import qc_state_invalidate
        qc_state_invalidate(self.state.h)

    def apply_1q(self, q, U):
        self.state.apply_1q(q, U)

    def apply_ctrl(self, c, t, U):
        self.state.apply_ctrl(c, t, U)

    def cnot(self, c, t):
        self.state.cnot(c, t)

    def cphase(self, c, t, k):
        self.state.cphase(c, t, k)

    def hadamard_layer(self, mask):
        self.state.apply_1q_layer(np.stack([H_MAT] * self.state.n), mask)

    def grover_partial(self, marked_local) -> complex:
        from . import qc_grover_partial
        return qc_grover_partial(self.state.h, marked_local)

    def grover_apply(self, marked_local, mean: complex):
        from . import qc_grover_apply_mean
        qc_grover_apply_mean(self.state.h, marked_local, mean)

    def norm2(self) -> float:
        return self.state.norm()

    def close(self):
        self.state.close()


# --------------------------------------------------------------- the state --

class ShardedState:
    """n logical qubits over comm.world = 2^p ranks (see the module text)."""

    def __init__(self, n: int, ops, comm):
        world = comm.world
        p = world.bit_length() - 1
        if (1 << p) != world:
            raise ValueError("the number of ranks must be a power of two (got %d)" % world)
        if n - p < 2:
            raise ValueError("need at least two local qubits per shard (n = %d, %d ranks)" % (n, world))
        self.n, self.p, self.nl = n, p, n - p
        self.ops, self.comm = ops, comm
        self.rank = comm.rank
        self.qmap = list(range(n))  # logical qubit -> physical bit
        self.exchanges = 0           # half-shard exchanges this rank took part in

    # -------------------------------------------------------- index maps --
    def physical(self, x: int) -> int:
        """Physical index of logical basis index x."""
        y = 0
        for t in range(self.n):
            if (x >> t) & 1:
                y |= 1 << self.qmap[t]
        return y

    def _rank_bit(self, ph: int) -> int:
        return (self.rank >> (ph - self.nl)) & 1

    # ------------------------------------------------------- the exchange --
    def _swap_with_top_local(self, g: int):
        """Swap global physical bit g with the top local bit L: the pairwise
        half-shard exchange with rank ^ 2^(g - nl)."""
        L = self.nl - 1
        d = g - self.nl
        partner = self.rank ^ (1 << d)
        b = (self.rank >> d) & 1
        half = 1 << L
        t = self.ops.tensor
        mine = t[(1 - b) * half:(2 - b) * half]  # amplitudes whose bit L differs from our bit g
        recv = mine.clone() if not hasattr(self, "_buf") or self._buf.shape != mine.shape else self._buf
        self._buf = recv
        self.comm.sendrecv(mine, recv, partner)
        mine.copy_(recv)
        self.ops.invalidate()
        self.exchanges += 1
        a = self.qmap.index(g)
        c = self.qmap.index(L)
        self.qmap[a], self.qmap[c] = L, g

    def _local(self, t: int) -> int:
        ph = self.qmap[t]
        if ph >= self.nl:
            self._swap_with_top_local(ph)
        return self.qmap[t]

    # ------------------------------------------------------- preparation --
    def reset(self, basis: int = 0):
        y = self.physical(int(basis))
        if (y >> self.nl) == self.rank:
            self.ops.zero(y & ((1 << self.nl) - 1))
        else:
            self.ops.zero(None)
        return self

    # ------------------------------------------------------------- gates --
    def apply_1q(self, t: int, U):
        self.ops.apply_1q(self._local(t), U)

    def apply_ctrl(self, c: int, t: int, U):
        pt = self._local(t)
        pc = self.qmap[c]
        if pc < self.nl:
            self.ops.apply_ctrl(pc, pt, U)
        elif self._rank_bit(pc):
            self.ops.apply_1q(pt, U)

    def cnot(self, c: int, t: int):
        pt = self._local(t)
        pc = self.qmap[c]
        if pc < self.nl:
            self.ops.cnot(pc, pt)
        elif self._rank_bit(pc):
            self.ops.apply_1q(pt, X_MAT)

    def cphase(self, c: int, t: int, k: int):
        """diag(1, 1, 1, e^{2 pi i / 2^k}) on (c, t) (Eq. cphasek): diagonal,
        so no amplitude moves between ranks."""
        pc, pt = self.qmap[c], self.qmap[t]
        ph = complex(math.cos(2 * math.pi / (1 << k)), math.sin(2 * math.pi / (1 << k)))
        if k == 1:
            ph = -1.0
        elif k == 2:
            ph = 1j
        P = np.array([[1, 0], [0, ph]], dtype=np.complex128)
        lc, lt = pc < self.nl, pt < self.nl
        if lc and lt:
            self.ops.cphase(pc, pt, k)
        elif lt:
            if self._rank_bit(pc):
                self.ops.apply_1q(pt, P)
        elif lc:
            if self._rank_bit(pt):
                self.ops.apply_1q(pc, P)
        elif self._rank_bit(pc) and self._rank_bit(pt):
            self.ops.apply_1q(0, np.array([[ph, 0], [0, ph]], dtype=np.complex128))

    def swap(self, a: int, b: int):
        self.qmap[a], self.qmap[b] = self.qmap[b], self.qmap[a]

    def hall(self):
        """H on every qubit: the local ones in one Hadamard layer, then each
        global one through the top local bit (whose qubit has had its H)."""
        mask = 0
        for t in range(self.n):
            if self.qmap[t] < self.nl:
                mask |= 1 << self.qmap[t]
        self.ops.hadamard_layer(mask)
        for t in range(self.n):
            if self.qmap[t] >= self.nl:
                self.ops.apply_1q(self._local(t), H_MAT)

    # ------------------------------------------------------------ Grover --
    def grover_step(self, marked):
        """G = HALL . Inv . HALL . Oracle (sec. 5.1) on the split state: the
        oracle flips the marked items on the ranks that hold them; the mean
        of the flipped state is one all-reduce of the shards' partial sums."""
        mask = (1 << self.nl) - 1
        loc = []
        for m in marked:
            y = self.physical(int(m))
            if (y >> self.nl) == self.rank:
                loc.append(y & mask)
        P = self.ops.grover_partial(loc)
        tot = self.comm.allreduce([P.real, P.imag], self._red_device())
        mean = complex(tot[0], tot[1]) / float(1 << self.n)
        self.ops.grover_apply(loc, mean)

    # --------------------------------------------------------------- QFT --
    def qft(self):
        """Appendix A's circuit: for j = n-1 .. 0, H on j and CPHASEK(j, t)
        with k = j - t + 1 for every t < j, then the qubit-order reversal as
        a relabelling.  Only the Hadamards of qubits on global bits need an
        exchange."""
        for j in range(self.n - 1, -1, -1):
            self.apply_1q(j, H_MAT)
            for t in range(j - 1, -1, -1):
                self.cphase(j, t, j - t + 1)
        self.qmap = [self.qmap[self.n - 1 - t] for t in range(self.n)]

    # -------------------------------------------------------- reductions --
    def _red_device(self):
        return getattr(self.ops, "device", "cpu")

    def norm2(self) -> float:
        return float(self.comm.allreduce([self.ops.norm2()], self._red_device())[0])

    def gather(self) -> np.ndarray:
        """The whole state in logical order (every rank gets it)."""
        parts = self.comm.allgather(self.ops.tensor)
        phys = np.concatenate([p.detach().cpu().numpy() for p in parts]).astype(np.complex128)
        N = 1 << self.n
        x = np.arange(N, dtype=np.int64)
        y = np.zeros(N, dtype=np.int64)
        for t in range(self.n):
            y |= ((x >> t) & 1) << self.qmap[t]
        return phys[y]
