"""Failure detection without a GPU fault: the Jacobi sweep limit and the
cross-CTA wait limit are set from the host so that they run out; the step
returns TNLBM_E_NOCONV / TNLBM_E_TIMEOUT, the simulation can be destroyed, and
the context stays usable for a fresh simulation.  No wait is left unbounded
and no kernel traps: the waits that run out here are bounded mbarrier polls
and the Jacobi simply stops after its last allowed sweep."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

E_TIMEOUT, E_NOCONV = -4, -5


@pytest.fixture(scope="module")
def tl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_07615_gb300 as pkg
    return pkg


def _channel(tl, prec, **kw):
    # rest start: the rounding at create sees rank-1 centres (no Jacobi pair)
    return tl.Sim(3, tau=0.8, periodic=(1, 1, 0), force=(1e-4, 0, 0), chi_max=16, eps=1e-10,
                  precision=prec, hadamard=0, **kw)


def _fresh_run_is_fine(tl, prec):
    sim = _channel(tl, prec)
    sim.step(2)
    rho, u = sim.macroscopic()
    assert np.isfinite(u).all() and sim.stats()["status"] == 0
    sim.close()


@pytest.mark.parametrize("prec", [1, 3])
def test_jacobi_sweep_limit_returns_noconv(tl, prec):
    from paper_2512_07615_gb300.native import TnlbmError
    sim = _channel(tl, prec)
    sim.step(1)
    sim.set_limits(jacobi_max_sweeps=1)
    with pytest.raises(TnlbmError) as ei:
        sim.step(1)
    assert ei.value.code == E_NOCONV
    assert "sweep limit" in str(ei.value)
    sim.close()
    _fresh_run_is_fine(tl, prec)


def test_cluster_wait_limit_returns_timeout(tl):
    """Mixed precision with two CTAs per rounding job: with a wait limit of
    1 ns the workers stop waiting for the leader (which is still in its QR
    sweep), record ST_TIMEOUT and leave through the exit barrier; the leader's
    next wait runs out in turn.  The step reports TNLBM_E_TIMEOUT."""
    from paper_2512_07615_gb300.native import TnlbmError
    sim = _channel(tl, 3, max_cluster=2)
    sim.step(1)
    sim.set_limits(wait_limit_ns=1)
    with pytest.raises(TnlbmError) as ei:
        sim.step(1)
    assert ei.value.code == E_TIMEOUT
    sim.close()
    _fresh_run_is_fine(tl, 3)
