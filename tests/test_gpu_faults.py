"""Failure detection through the C ABI, with every failure made on the host
side or by a bounded wait that is made to run out (no GPU is faulted, trapped
or hung):

* a tensor-core pipeline wait that runs out (a barrier that nothing arrives
  at, given up after 1 ms) -> TTN_ERR_TIMEOUT, from a bare contraction and
  from a TDVP step; the context works again once its state is reloaded;
* the Krylov dimension capped at 2 -> TTN_ERR_KRYLOV;
* a NaN node tensor set from the host -> TTN_ERR_NUMERIC at the next step;
* an allocation made to fail -> TTN_ERR_ALLOC, at creation and when a
  workspace grows.
"""
import os
import tempfile

import numpy as np
import pytest

from paper_2210_03763_gb300 import workloads as W

pytestmark = pytest.mark.gpu
ARG, ALLOC, KRYLOV, NUMERIC, TIMEOUT = 1, 2, 4, 5, 6


@pytest.fixture(scope="module")
def native():
    import __graft_entry__ as g
    g.build()
    from paper_2210_03763_gb300 import native as nat
    yield nat
    nat.inject(nat.INJECT_NONE)


@pytest.fixture(autouse=True)
def clear_hooks(native):
    native.inject(native.INJECT_NONE)
    yield
    native.inject(native.INJECT_NONE)


def _ctx(native, Lx, Ly, chi, prec, seed=3):
    g = native.TTN(Lx, Ly, chi)
    g.set_precision(prec)
    g.set_hamiltonian(W.square_lattice(Lx, Ly), 20.0)
    g.apply_pulse(W.random_constant_schedule(Lx * Ly, seed))
    g.set_product_state(W.random_product_amps(Lx * Ly, seed + 1))
    return g


def test_inject_rejects_bad_hooks(native):
    with pytest.raises(native.TTNError) as e:
        native.inject(9, 1)
    assert e.value.code == ARG
    with pytest.raises(native.TTNError):
        native.inject(native.INJECT_KRYLOV_MMAX, 31)


def test_contraction_timeout_is_reported_and_cleared(native):
    rng = np.random.default_rng(0)
    A = rng.normal(size=(256, 128)) + 1j * rng.normal(size=(256, 128))
    B = rng.normal(size=(128, 192)) + 1j * rng.normal(size=(128, 192))
    native.inject(native.INJECT_TC_STALL, 1)
    with pytest.raises(native.TTNError) as e:
        native.contract_host(A, B, native.SPLIT_TF32X3)
    assert e.value.code == TIMEOUT
    # the hook is spent: the next contraction runs normally
    C, tc, _ = native.contract_host(A, B, native.SPLIT_TF32X3)
    assert tc and np.max(abs(C - A @ B)) < 1e-6 * np.max(abs(A @ B))


def test_step_timeout_then_reload(native):
    g = _ctx(native, 4, 4, 64, native.SPLIT_TF32X3)
    g.step(0.02)
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "s.ttn")
        g.save(path)
        native.inject(native.INJECT_TC_STALL, 1)
        with pytest.raises(native.TTNError) as e:
            g.step(0.02)
        assert e.value.code == TIMEOUT
        native.inject(native.INJECT_NONE)
        g.load(path)
        g.step(0.02)
        ref = _ctx(native, 4, 4, 64, native.SPLIT_TF32X3)
        ref.load(path)
        ref.step(0.02)
        F = g.fidelity(ref)
        assert abs(1 - F / (g.norm() * ref.norm())) < 1e-12
        assert abs(g.time() - ref.time()) == 0.0
        ref.close()
    g.close()


def test_krylov_cap_reports_krylov_error(native):
    g = _ctx(native, 2, 2, 16, native.FP64)
    native.inject(native.INJECT_KRYLOV_MMAX, 2)
    with pytest.raises(native.TTNError) as e:
        g.step(0.5)
    assert e.value.code == KRYLOV
    g.close()


def test_nan_node_reports_numeric_error(native):
    g = _ctx(native, 2, 2, 16, native.FP64)
    X = g.get_node(0)
    X[1, 1, 0] = np.nan
    g.set_node(0, X)
    with pytest.raises(native.TTNError) as e:
        g.step(0.02)
    assert e.value.code == NUMERIC
    g.close()


def test_allocation_failure(native):
    native.inject(native.INJECT_ALLOC_FAIL, 1)
    with pytest.raises(native.TTNError) as e:
        native.TTN(2, 2, 16)
    assert e.value.code == ALLOC
    # a workspace that grows inside a step: the split-precision workspace of a
    # fresh context is allocated at its first tensor-core contraction
    g = _ctx(native, 4, 4, 64, native.SPLIT_TF32X3)
    native.inject(native.INJECT_ALLOC_FAIL, 1)
    with pytest.raises(native.TTNError) as e:
        g.step(0.02)
    assert e.value.code == ALLOC
    g.close()
    native.inject(native.INJECT_NONE)
    h = native.TTN(2, 2, 16)   # allocations work again
    h.close()
