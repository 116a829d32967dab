"""The algebra a multi-GPU sub-iteration would rest on, checked on the CPU
with the FP64 oracle (paper Eqs. 7-8).

The events of a subset are independent in the E-step: split them into K
shards, and each shard's partial back-projection b^k_n = sum_{j in shard k}
p_jn / y_j sums to the full b_n.  One all-reduce of b (N_nz values) per
sub-iteration then gives every rank the same update f_n b_n / (T s^i_n).
This build runs replicas only (no run here uses more than one GPU), so no
exchange is built; these tests pin the algebra such a shard would use: the
partial sums in one process, and two gloo ranks whose all-reduced partials
reproduce the single-process OSEM iterates."""
import os
import socket
import sys

import numpy as np

import oracle
from paper_2002_12471_gb300 import synthetic as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _case():
    ph, g, J, ns, ni = S.workload("tiny16")
    ev = S.simulate_events(ph, g, J, seed=21)
    P = oracle.Problem(dict(g, pixel_mm=ph.pixel_mm), ph.mu)
    p = P.model(ev.angle, ev.u_mm, ev.e_kev)
    s = P.sensitivity(ns)
    return p, ev.angle, s, ns, ni, J


def _backprojection(p_rows, f):
    y = p_rows @ f
    ok = y > 0
    return p_rows[ok].T @ (1.0 / y[ok])


def _sharded_osem(p, angle, s, n_iters, f0, T, shards, allreduce):
    """OSEM where the rows of every subset are split over `shards` (lists of
    event indices) and the partial back-projections are summed by
    `allreduce` before the update."""
    sub = oracle.subset_of(angle, s.shape[0])
    f = np.array(f0, dtype=np.float64)
    for _ in range(n_iters):
        for i in range(s.shape[0]):
            parts = [_backprojection(p[sh[sub[sh] == i]], f) for sh in shards]
            b = allreduce(parts)
            pos = s[i] > 0
            out = np.zeros_like(f)
            out[pos] = f[pos] * b[pos] / (T * s[i][pos])
            f = out
    return f


def test_shard_partials_sum_to_the_full_backprojection_and_osem():
    p, angle, s, ns, ni, J = _case()
    T = 1.7
    f0 = oracle.initial_image(J, s.sum(0), T)
    rng = np.random.default_rng(3)
    for K in (2, 3, 5):
        owner = rng.integers(0, K, len(angle))          # uneven shards
        shards = [np.nonzero(owner == k)[0] for k in range(K)]
        b_full = _backprojection(p, f0)
        b_sum = np.sum([_backprojection(p[sh], f0) for sh in shards], axis=0)
        np.testing.assert_allclose(b_sum, b_full, rtol=1e-12, atol=1e-300)
        f_ref, _ = oracle.osem(p, angle, s, ni, f0, T)
        f_sh = _sharded_osem(p, angle, s, ni, f0, T, shards, lambda parts: np.sum(parts, axis=0))
        assert oracle.rel_l2(f_sh, f_ref) <= 1e-12


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, angle, s, ns, ni, J = _case()
        T = 1.0
        f0 = oracle.initial_image(J, s.sum(0), T)
        mine = np.arange(rank, len(angle), world)     # this rank's events

        def allreduce(parts):
            b = torch.from_numpy(np.asarray(parts[0], dtype=np.float64).copy())
            dist.all_reduce(b, op=dist.ReduceOp.SUM)
            return b.numpy()

        f = _sharded_osem(p, angle, s, ni, f0, T, [mine], allreduce)
        out.put((rank, f))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_with_all_reduced_partials_match_single_process_osem():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = dict(q.get(timeout=300) for _ in range(2))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p, angle, s, ns, ni, J = _case()
    f_ref, _ = oracle.osem(p, angle, s, ni, oracle.initial_image(J, s.sum(0), 1.0), 1.0)
    for r in range(2):
        assert oracle.rel_l2(res[r], f_ref) <= 1e-12
    np.testing.assert_array_equal(res[0], res[1])
