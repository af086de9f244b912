"""Subtree decomposition of Algorithm 2 over ranks, on CPU with gloo (world size 2).

Below the root, Algorithm 2 touches only a node's own blocks and its children's, so the levels
L..1 of the subtree under each level-1 node are independent: each rank sweeps its subtree and
sends the r rows it contributes to the root's reduced test and sample blocks
(Eq. omega_tau_and_y_tau) together with its factors; rank 0 finishes the root
(D = Y Omega^+). The gathered result must equal the single-process sweep bit for bit.
The node arithmetic is the oracle's; this test covers the decomposition and the exchange.
"""

import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from hbs_inputs import exact_hbs
from oracle import compress as oc
from oracle.philox import gaussian_test_matrices
from oracle.tree import build_tree, children, level_nodes

N, K, R, S, LEAF, SEED = 400, 5, 8, 24, 16, 3


def inputs():
    A = exact_hbs(N, LEAF, K, 1).dense()
    Om, Ps = gaussian_test_matrices(N, S, SEED)
    return Om, Ps, A @ Om, A.T @ Ps


def sweep_subtree(top, Om, Ps, Y, Z):
    """Levels L..1 of the subtree rooted at level-1 node ``top``; returns its factors and the
    node's contribution to the root's blocks."""
    L, off, size = build_tree(N, LEAF)
    U, V, D, blk = {}, {}, {}, {"Om": {}, "Ps": {}, "Y": {}, "Z": {}}
    for level in range(L, 0, -1):
        first = top << (level - 1)
        for t in range(first, first + (1 << (level - 1))):
            if level == L:
                rows = slice(off[t], off[t] + size[t])
                blk["Om"][t], blk["Ps"][t], blk["Y"][t], blk["Z"][t] = Om[rows], Ps[rows], Y[rows], Z[rows]
            else:
                a, b = children(t)
                (blk["Om"][t], blk["Ps"][t], blk["Y"][t], blk["Z"][t]) = oc.merge(
                    blk["Om"], blk["Ps"], blk["Y"], blk["Z"], U, V, D, a, b)
            U[t], V[t], D[t] = oc.node_step(blk["Om"][t], blk["Ps"][t], blk["Y"][t], blk["Z"][t], R)
    t = top
    contrib = (V[t].T @ blk["Om"][t], U[t].T @ blk["Ps"][t],
               U[t].T @ (blk["Y"][t] - D[t] @ blk["Om"][t]), V[t].T @ (blk["Z"][t] - D[t].T @ blk["Ps"][t]))
    return U, V, D, contrib


def worker(rank, world, port, queue):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        Om, Ps, Y, Z = inputs()
        U, V, D, contrib = sweep_subtree(2 + rank, Om, Ps, Y, Z)
        gathered = [None] * world if rank == 0 else None
        dist.gather_object((rank, U, V, D, contrib), gathered, dst=0)
        if rank == 0:
            parts = dict((g[0], g[1:]) for g in gathered)
            Uall, Vall, Dall = {}, {}, {}
            for g in range(world):
                Uall.update(parts[g][0])
                Vall.update(parts[g][1])
                Dall.update(parts[g][2])
            root = [np.vstack([parts[0][3][j], parts[1][3][j]]) for j in range(4)]
            Dall[1] = root[2] @ oc.pinv(root[0])
            queue.put((Uall, Vall, Dall))
    finally:
        dist.destroy_process_group()


def free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def test_subtree_decomposition_over_two_gloo_ranks_is_exact():
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = free_port()
    procs = mp.start_processes(worker, args=(2, port, queue), nprocs=2, join=False,
                               start_method="spawn")
    U, V, D = queue.get(timeout=240)   # read before joining: the result does not fit in a pipe
    while not procs.join(timeout=60):
        pass
    F = oc.compress(*inputs(), R, LEAF)
    assert set(D) == set(F.D) and set(U) == set(F.U)
    for t in F.D:
        assert np.array_equal(D[t], F.D[t])
        if t > 1:
            assert np.array_equal(U[t], F.U[t]) and np.array_equal(V[t], F.V[t])
