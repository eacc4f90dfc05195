"""Groups (mace_group_*): the Mann iterations of several states with
different geometries advanced together, the ICD passes of all of them in one
queue-fed launch per pass.  Each member must follow the iterates it has alone
(Algorithm 1 per member) and converge to its own MAP image."""
import numpy as np
import pytest

import oracle
import synth
from helpers import nrmse

pytestmark = pytest.mark.gpu

# (nx, ny, views, channels, agents, view partition seed or None, batch):
# a ragged image with uneven agents, many small agents, and agents with 150
# views each (the variant that decodes each column as it is used)
CASES = [(45, 38, 40, 61, 3, 7, 1), (32, 32, 64, 47, 16, None, 2), (40, 40, 300, 59, 2, None, 1)]


def _case(k):
    nx, ny, V, D, N, pseed, B = CASES[k]
    va = None if pseed is None else synth.uneven_partition(pseed, V, N, 10, 16)
    m = min(nx, ny)
    p = synth.sinogram(synth.ellipses(31 + k, m, 0.02 * 64 / m), V, D)
    ys, ls = zip(*[synth.measurements(p, 2e4, synth.CounterRNG(171 + 10 * k + b)) for b in range(B)])
    y, lam = np.stack(ys), np.stack(ls)
    sx = synth.prior_sigma_x(lam[0], V, frac=1.0)
    return dict(nx=nx, ny=ny, V=V, D=D, N=N, va=va, B=B, y=y, lam=lam, sx=sx)


def _params(mace, c, **kw):
    a = dict(prior="qggmrf", sigma_x=c["sx"], sigma=0.2, sigma_mode=1, rho=0.8, sweeps_per_iter=2, symmetric=True,
             recompute_every=10, tol=1e-7, max_iter=6000, concurrency=2, schedule=1)
    a.update(kw)
    return mace.make_params(**a)


@pytest.fixture(scope="module")
def members(gpu_lib):
    mace = gpu_lib
    cs = [_case(k) for k in range(len(CASES))]
    sms = [mace.mace_build_sysmatrix(c["nx"], c["ny"], c["V"], c["D"], c["N"], view_agent=c["va"], sv_size=4)
           for c in cs]
    yield mace, cs, sms
    for sm in sms:
        sm.close()


def test_group_follows_each_member_alone(members):
    """Concurrency 1 (each item a whole (reconstruction, agent) pair, so no
    two warps share an error sinogram): 20 iterations in the group give the
    iterates of each member run alone, to float rounding."""
    import torch
    mace, cs, sms = members
    alone = []
    for c, sm in zip(cs, sms):
        st = mace.mace_init(sm, c["y"], c["lam"], _params(mace, c, concurrency=1), batch=c["B"])
        st.iterate(20)
        alone.append(st.get_state())
        st.close()
    s = torch.cuda.Stream()
    sts = [mace.mace_init(sm, c["y"], c["lam"], _params(mace, c, concurrency=1), batch=c["B"])
           for c, sm in zip(cs, sms)]
    with mace.mace_group_create(sts, stream=s) as grp:
        grp.launch(20)
        for k, st in enumerate(sts):
            st.poll()
            assert st.stats()["iters"] == 20
            w, X = st.get_state()
            w0, X0 = alone[k]
            dw = float(np.abs(w - w0).max() / np.abs(w0).max())
            dX = float(np.abs(X - X0).max() / np.abs(X0).max())
            print("member %d: max relative difference w %.1e X %.1e" % (k, dw, dX))
            assert dw < 1e-5 and dX < 1e-5
    for st in sts:
        st.close()


def test_group_members_converge_to_their_map(members):
    """Two items per pair, the group launched in chunks until every
    member has converged: each reconstruction equals the oracle's MAP image
    of its own scan."""
    import torch
    mace, cs, sms = members
    s = torch.cuda.Stream()
    sts = [mace.mace_init(sm, c["y"], c["lam"], _params(mace, c), batch=c["B"]) for c, sm in zip(cs, sms)]
    grp = mace.mace_group_create(sts, stream=s)
    done = [False] * len(sts)
    for chunk in range(600):
        grp.launch(10)
        polls = []
        for k, st in enumerate(sts):
            try:
                polls.append(st.poll())
            except mace.MaceError:
                print("member %d failed at iteration %d" % (k, 10 * (chunk + 1)))
                raise
        if chunk % 50 == 0:
            print("iteration %d: residuals %s" % (10 * (chunk + 1), " ".join("%.2e" % r for r, _ in polls)))
        done = [c for _, c in polls]
        if all(done):
            break
    grp.close()
    assert all(done)
    for c, st in zip(cs, sts):
        x = np.asarray(st.consensus(), np.float64).reshape(c["B"], -1)
        for b in range(c["B"]):
            P = oracle.Problem(c["nx"], c["ny"], c["V"], c["D"], c["y"][b], c["lam"][b], n_agents=c["N"],
                               view_agent=c["va"], prior="qggmrf", sigma_x=c["sx"])
            xs, _, _ = P.central_icd(max_sweeps=40000, tol=1e-13)
            err = nrmse(x[b], xs)
            print("%dx%d, %d agents: iters %d, NRMSE vs oracle %.2e" % (c["nx"], c["ny"], c["N"],
                                                                       st.stats()["iters"], err))
            assert err < 1e-4
        st.close()


def test_group_rejects_fixed_schedule_and_duplicates(members):
    mace, cs, sms = members
    c, sm = cs[0], sms[0]
    a = mace.mace_init(sm, c["y"], c["lam"], _params(mace, c), batch=c["B"])
    b = mace.mace_init(sm, c["y"], c["lam"], _params(mace, c, schedule=0), batch=c["B"])
    for bad in ([a, b], [a, a]):
        with pytest.raises(mace.MaceError) as ei:
            mace.mace_group_create(bad)
        assert ei.value.code == mace.MACE_EINVAL
    a.close()
    b.close()


def test_group_diverging_member_is_isolated(members):
    """A member whose iteration diverges (normalised sigma 10 with one
    forward pass: outside Theorem 2's range) fills its error sinogram with
    non-finite values while it shares launches with a well-posed member; it
    is reported (MACE_ENUMERIC), dropped from the group, and the other
    member still converges to its oracle MAP image."""
    import torch
    mace, cs, sms = members
    c = cs[0]
    bad = mace.mace_init(sms[0], c["y"], c["lam"], _params(mace, c, sigma=10.0, sweeps_per_iter=1, symmetric=False,
                                                             concurrency=-1), batch=c["B"])
    good = mace.mace_init(sms[0], c["y"], c["lam"], _params(mace, c), batch=c["B"])
    grp = mace.mace_group_create([bad, good], stream=torch.cuda.Stream())
    failed_at = None
    for chunk in range(100):
        grp.launch(10)
        try:
            bad.poll()
        except mace.MaceError as e:
            assert e.code == mace.MACE_ENUMERIC
            failed_at = 10 * (chunk + 1)
            break
    assert failed_at is not None
    grp.update([good])
    bad.close()
    conv = False
    for _ in range(600):
        grp.launch(10)
        r, conv = good.poll()
        if conv:
            break
    grp.close()
    assert conv
    x = np.asarray(good.consensus(), np.float64).ravel()
    good.close()
    P = oracle.Problem(c["nx"], c["ny"], c["V"], c["D"], c["y"][0], c["lam"][0], n_agents=c["N"],
                       view_agent=c["va"], prior="qggmrf", sigma_x=c["sx"])
    xs, _, _ = P.central_icd(max_sweeps=40000, tol=1e-13)
    err = nrmse(x, xs)
    print("diverged member reported after %d iterations; the other: NRMSE vs oracle %.2e" % (failed_at, err))
    assert np.all(np.isfinite(x)) and err < 1e-4
