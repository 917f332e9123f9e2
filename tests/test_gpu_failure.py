"""Error paths of the device-side waits and of the line factorisation, made to happen on the
host side only: a bounded mbarrier wait of the factor or sweep kernels is given a try limit of
zero (helm_set_wait_tries), so that it gives up at once; the kernel then stops every CTA of its
cluster, drains, returns, and the call reports HELM_ETIMEOUT.  The context stays usable: the
next call with the default limit gives the same result as before.  A model with a NaN value
(a corrupted input copy) makes a pivot non-finite, which the factor reports as
HELM_ESINGULAR.  The host-side fault injection (HELM_FAULT=alloc|pivot|timeout|nan_rhs) drives
ENOMEM, ESINGULAR, ETIMEOUT and ENOCONV through the library's own paths, and the calls after it
are unaffected."""
import numpy as np
import pytest
import torch

hm = pytest.importorskip("paper_2301_10762_gb300.helm")

pytestmark = pytest.mark.gpu

ENOMEM, ENOCONV, ESINGULAR, ETIMEOUT = 2, 4, 5, 6


@pytest.fixture(autouse=True)
def default_wait_limit():
    yield
    hm.helm_set_wait_tries(-1)


def _case(nx, nz, nrhs, seed=9):
    rng = np.random.default_rng(seed)
    c = 1.0 + 0.5 * rng.uniform(0, 1, (nx, nz))
    m = (1.0 / c ** 2).reshape(-1)
    om = np.array([6.0, 11.0])
    B = rng.standard_normal((2, nrhs, nx * nz)) + 1j * rng.standard_normal((2, nrhs, nx * nz))
    return m, om, torch.tensor(B, device="cuda")


def _same(X, ref, prec):
    """The FP64 path is bitwise reproducible; the mixed path may stop its refinement one sweep
    apart (its residual norms are summed by atomics), so it is compared at its own tolerance."""
    torch.cuda.synchronize()
    if prec == hm.HELM_FP64:
        assert torch.equal(X, ref)
    else:
        err = torch.linalg.vector_norm(X - ref, dim=-1) / torch.linalg.vector_norm(ref, dim=-1)
        assert float(err.max()) <= 1e-10


SHAPES = [(48, 40, 3), (64, 64, 8)]   # clusters of 4 / 8 CTAs; FMA and tensor-pipe products


@pytest.mark.parametrize("prec", [hm.HELM_FP64, hm.HELM_MIXED])
@pytest.mark.parametrize("shape", SHAPES)
def test_sweep_wait_gives_up_with_etimeout_and_the_context_survives(prec, shape):
    nx, nz, nrhs = shape
    m, om, B = _case(nx, nz, nrhs)
    op = hm.helm_assemble(nx, nz, 1.0, 1.0, torch.tensor(m, device="cuda"), om)
    f = hm.helm_factor(op, prec)
    ref, _ = hm.helm_solve(f, B, rtol=1e-12, max_iter=10)
    hm.helm_set_wait_tries(0)
    for solve in (hm.helm_solve, hm.helm_adjoint_solve):
        with pytest.raises(hm.HelmError) as e:
            solve(f, B, rtol=1e-12, max_iter=10)
        assert e.value.status == ETIMEOUT
    hm.helm_set_wait_tries(-1)
    X, info = hm.helm_solve(f, B, rtol=1e-12, max_iter=10)
    _same(X, ref, prec)
    if prec == hm.HELM_MIXED:
        assert info["max_relres"] <= 1e-12


@pytest.mark.parametrize("prec", [hm.HELM_FP64, hm.HELM_MIXED])
@pytest.mark.parametrize("shape", SHAPES)
def test_factor_wait_gives_up_with_etimeout_and_the_context_survives(prec, shape):
    nx, nz, nrhs = shape
    m, om, B = _case(nx, nz, nrhs)
    op = hm.helm_assemble(nx, nz, 1.0, 1.0, torch.tensor(m, device="cuda"), om)
    f0 = hm.helm_factor(op, prec)
    ref, _ = hm.helm_solve(f0, B, rtol=1e-12, max_iter=10)
    f0.close()
    hm.helm_set_wait_tries(0)
    with pytest.raises(hm.HelmError) as e:
        hm.helm_factor(op, prec)
    assert e.value.status == ETIMEOUT
    hm.helm_set_wait_tries(-1)
    f = hm.helm_factor(op, prec)
    X, _ = hm.helm_solve(f, B, rtol=1e-12, max_iter=10)
    _same(X, ref, prec)


@pytest.mark.parametrize("prec", [hm.HELM_FP64, hm.HELM_MIXED])
def test_non_finite_model_value_is_reported_as_esingular(prec):
    nx, nz = 48, 40
    m, om, _ = _case(nx, nz, 1)
    for node in (0, nz * (nx // 2) + nz // 3):   # first line of the left team; a middle line
        bad = m.copy()
        bad[node] = np.nan
        op = hm.helm_assemble(nx, nz, 1.0, 1.0, torch.tensor(bad, device="cuda"), om)
        with pytest.raises(hm.HelmError) as e:
            hm.helm_factor(op, prec)
        assert e.value.status == ESINGULAR
        op.close()
    # a clean model on the same context still factors
    op = hm.helm_assemble(nx, nz, 1.0, 1.0, torch.tensor(m, device="cuda"), om)
    hm.helm_factor(op, prec).close()


def test_fault_alloc_gives_enomem_and_nothing_sticks(monkeypatch):
    nx, nz, nrhs = 48, 40, 3
    m, om, B = _case(nx, nz, nrhs)
    md = torch.tensor(m, device="cuda")
    op = hm.helm_assemble(nx, nz, 1.0, 1.0, md, om)
    f = hm.helm_factor(op, hm.HELM_MIXED)
    ref, _ = hm.helm_solve(f, B, rtol=1e-12, max_iter=10)
    monkeypatch.setenv("HELM_FAULT", "alloc")
    assert hm.helm_fault_mask() == hm.HELM_FAULT_ALLOC
    for call in (lambda: hm.helm_assemble(nx, nz, 1.0, 1.0, md, om), lambda: hm.helm_factor(op, hm.HELM_FP64),
                 lambda: hm.helm_factor(op, hm.HELM_MIXED, method=hm.HELM_FACTOR_BCR)):
        with pytest.raises(hm.HelmError) as e:
            call()
        assert e.value.status == ENOMEM
    monkeypatch.delenv("HELM_FAULT")
    X, _ = hm.helm_solve(f, B, rtol=1e-12, max_iter=10)
    _same(X, ref, hm.HELM_MIXED)


@pytest.mark.parametrize("prec,method", [(hm.HELM_FP64, hm.HELM_FACTOR_AUTO), (hm.HELM_MIXED, hm.HELM_FACTOR_LINE),
                                         (hm.HELM_MIXED, hm.HELM_FACTOR_BCR)])
def test_fault_pivot_gives_esingular_and_leaves_the_op_intact(monkeypatch, prec, method):
    nx, nz, nrhs = 48, 40, 3
    m, om, B = _case(nx, nz, nrhs)
    op = hm.helm_assemble(nx, nz, 1.0, 1.0, torch.tensor(m, device="cuda"), om)
    f0 = hm.helm_factor(op, prec, method=method)
    ref, _ = hm.helm_solve(f0, B, rtol=1e-12, max_iter=10)
    f0.close()
    monkeypatch.setenv("HELM_FAULT", "pivot")
    with pytest.raises(hm.HelmError) as e:
        hm.helm_factor(op, prec, method=method)
    assert e.value.status == ESINGULAR
    monkeypatch.delenv("HELM_FAULT")
    f = hm.helm_factor(op, prec, method=method)
    X, _ = hm.helm_solve(f, B, rtol=1e-12, max_iter=10)
    _same(X, ref, prec)


def test_fault_timeout_gives_etimeout(monkeypatch):
    nx, nz, nrhs = 64, 64, 8
    m, om, B = _case(nx, nz, nrhs)
    op = hm.helm_assemble(nx, nz, 1.0, 1.0, torch.tensor(m, device="cuda"), om)
    f = hm.helm_factor(op, hm.HELM_FP64)
    ref, _ = hm.helm_solve(f, B, rtol=1e-12, max_iter=10)
    monkeypatch.setenv("HELM_FAULT", "timeout")
    with pytest.raises(hm.HelmError) as e:
        hm.helm_factor(op, hm.HELM_FP64)
    assert e.value.status == ETIMEOUT
    with pytest.raises(hm.HelmError) as e:
        hm.helm_solve(f, B, rtol=1e-12, max_iter=10)
    assert e.value.status == ETIMEOUT
    monkeypatch.delenv("HELM_FAULT")
    X, _ = hm.helm_solve(f, B, rtol=1e-12, max_iter=10)
    _same(X, ref, hm.HELM_FP64)


@pytest.mark.parametrize("prec", [hm.HELM_FP64, hm.HELM_MIXED])
def test_fault_nan_rhs_gives_enoconv_and_leaves_b_intact(monkeypatch, prec):
    nx, nz, nrhs = 48, 40, 3
    m, om, B = _case(nx, nz, nrhs)
    op = hm.helm_assemble(nx, nz, 1.0, 1.0, torch.tensor(m, device="cuda"), om)
    f = hm.helm_factor(op, prec)
    ref, _ = hm.helm_solve(f, B, rtol=1e-12, max_iter=10)
    B0 = B.clone()
    monkeypatch.setenv("HELM_FAULT", "nan_rhs")
    for solve in (hm.helm_solve, hm.helm_adjoint_solve):
        with pytest.raises(hm.HelmError) as e:
            solve(f, B, rtol=1e-12, max_iter=10)
        assert e.value.status == ENOCONV
    monkeypatch.delenv("HELM_FAULT")
    assert torch.equal(B, B0)
    X, _ = hm.helm_solve(f, B, rtol=1e-12, max_iter=10)
    _same(X, ref, prec)
