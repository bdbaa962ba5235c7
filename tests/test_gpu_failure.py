"""The failure path of the bounded device waits, made to run out on purpose
without faulting or hanging anything.

jac_inject_stall gives the next sweep launch a grid-barrier target between
sweeps that no CTA ever reaches, and a wait limit of a few milliseconds.
The state producer's barrier wait then gives up, every CTA drains its own
copies and exits, and the launch ends with the workspace error word set:
the residual written is NaN, jac_sync and jac_residual report JAC_ETIMEOUT
and clear the word, and the same context then sweeps normally again (the
result checked against the oracle).  This is the library's counterpart of
the offload search's measurement time limit (Section 5.1.2)."""
import numpy as np
import pytest

import jacobi_inputs as ji
from _util import TOL, oracle_ref, rel_g, rel_p

pytestmark = pytest.mark.gpu
WAIT_NS = 2_000_000          # 2 ms: far above any legitimate wait on these grids


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_12115_gb300 import _build
    _build.build()
    import paper_2002_12115_gb300 as p
    return p


@pytest.mark.parametrize("prec,dims,owned", [("f32", (70, 21, 19), False), ("bf16", (131, 9, 12), True),
                                             ("f64", (37, 33, 29), False)])
def test_stalled_barrier_times_out_and_context_recovers(pkg, prec, dims, owned):
    I, J, K = dims
    n = 4
    f = ji.himeno_fields(I, J, K, seed=300 + I)
    with pkg.Jacobi(I, J, K, prec, owned=owned) as jac:
        jac.upload(f)
        jac.inject_stall(WAIT_NS)
        jac.sweep(n)
        p_out = np.zeros((K, J, I))
        res = np.zeros(1)
        jac.download_async(p_out, res)
        with pytest.raises(pkg.JacError) as err:
            jac.sync()
        assert err.value.status == 5                      # JAC_ETIMEOUT
        assert np.isnan(res[0])                           # the launch wrote NaN, not stale partials
        jac.sync()                                        # the error word was cleared

        # the residual route reports it too
        jac.upload(f)
        jac.inject_stall(WAIT_NS)
        jac.sweep(n)
        with pytest.raises(pkg.JacError) as err:
            jac.residual()
        assert err.value.status == 5

        # and the context sweeps normally afterwards
        jac.upload(f)
        jac.sweep(n)
        g = jac.residual()
        p = jac.download()
    op, og = oracle_ref(f, n, prec)
    assert rel_p(p, op) <= TOL[prec] and rel_g(g, og) <= TOL[prec], (rel_p(p, op), rel_g(g, og))


def test_single_sweep_launch_has_no_barrier_to_stall(pkg):
    """One sweep per launch never waits on the grid barrier: the injection
    is consumed and the result is normal."""
    I, J, K = 40, 17, 11
    f = ji.himeno_fields(I, J, K, seed=333)
    with pkg.Jacobi(I, J, K, "f32") as jac:
        jac.upload(f)
        jac.inject_stall(WAIT_NS)
        jac.sweep(1)
        g = jac.residual()
        p = jac.download()
    op, og = oracle_ref(f, 1, "f32")
    assert rel_p(p, op) <= TOL["f32"] and rel_g(g, og) <= TOL["f32"]
