"""Multi-rank path on CPU: world_size 2 over gloo.  Each rank computes the hypergradient
of its share of the training models (here with the CPU oracle standing in for the GPU
library) and the ranks assemble the average with one all-reduce; rank 0 checks it against
the single-process average over all models."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2301_10762_gb300.distributed import shard_models


def _models():
    import workloads as W
    out = []
    for k, (nx, nz) in enumerate([(10, 9), (12, 10), (9, 11)]):
        mt = W.layered_velocity(nx, nz, 50 + k)
        mf = W.gaussian_smooth(mt.reshape(nx, nz), 1.5).reshape(-1)
        out.append((nx, nz, mf, mt))
    return out


SRC = np.array([[0.0, 0.3], [0.0, 0.7]])
REC = np.array([[1.0, 0.25], [1.0, 0.6], [0.95, 0.8]])
OM = np.array([3.0, 6.0])


def _oracle_compute(models):
    from oracle import helmholtz as H
    acc = {"psi": 0.0, "dpsi_dalpha": 0.0, "dpsi_dp": np.zeros((3, 2)), "dpsi_dw": np.zeros(3)}
    for nx, nz, mf, mt in models:
        o = H.hypergradient(H.Grid(nx, nz), mf, mt, OM, SRC, REC, 1e-3, 1e-3, 1e-2, cg_fixed_iters=4)
        for k in acc:
            acc[k] = acc[k] + o[k] / len(models)
    return acc


def _worker(rank, world, port, out_path):
    import torch.distributed as dist
    from paper_2301_10762_gb300.distributed import distributed_hypergrad
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = distributed_hypergrad(_models(), _oracle_compute, n_rec=3)
    if rank == 0:
        np.savez(out_path, psi=res["psi"], dalpha=res["dpsi_dalpha"], dp=res["dpsi_dp"], dw=res["dpsi_dw"])
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_models_covers_every_model_once():
    for n, w in ((32, 8), (3, 2), (5, 4), (1, 3)):
        got = sorted(i for r in range(w) for i in shard_models(n, w, r))
        assert got == list(range(n))


def test_two_rank_gloo_hypergradient_equals_single_process(tmp_path):
    out = str(tmp_path / "res.npz")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    got = np.load(out)
    ref = _oracle_compute(_models())
    assert np.isclose(float(got["psi"]), ref["psi"], rtol=1e-13)
    assert np.isclose(float(got["dalpha"]), ref["dpsi_dalpha"], rtol=1e-12)
    assert np.allclose(got["dp"], ref["dpsi_dp"], rtol=1e-12, atol=1e-14)
    assert np.allclose(got["dw"], ref["dpsi_dw"], rtol=1e-12, atol=1e-14)


def test_four_ranks_three_models_one_rank_idle(tmp_path):
    """More ranks than models: the rank without a model contributes zeros to the all-reduce and
    the average is still the single-process one."""
    out = str(tmp_path / "res4.npz")
    mp.start_processes(_worker, args=(4, _free_port(), out), nprocs=4, start_method="spawn")
    got = np.load(out)
    ref = _oracle_compute(_models())
    assert np.isclose(float(got["psi"]), ref["psi"], rtol=1e-13)
    assert np.isclose(float(got["dalpha"]), ref["dpsi_dalpha"], rtol=1e-12)
    assert np.allclose(got["dp"], ref["dpsi_dp"], rtol=1e-12, atol=1e-14)
    assert np.allclose(got["dw"], ref["dpsi_dw"], rtol=1e-12, atol=1e-14)
