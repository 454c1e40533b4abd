"""Continuous-batching server, in both modes (one stream per slot, and the
lockstep group whose Arnoldi steps share launches): every result is the same
bits alone and in a mixed batch; admission by device footprint; faults stay
per request."""
import numpy as np
import pytest

from paper_2604_23265_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _mix(count, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        I = int(rng.choice([16, 24, 32]))
        M = int(rng.choice([8, 16]))
        md = W.grf_diffusive(seed * 100 + i, I=I, M=M, eps=float(np.exp(rng.uniform(np.log(1e-2), 0))),
                             g=float(rng.uniform(0, 0.8)))
        out.append(md)
    return out


def _lone(md, tol=1e-8):
    from paper_2604_23265_gb300 import rte
    ctx = rte.Context.from_medium(md)
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    info = ctx.solve(x, tol=tol)
    psi = torch.zeros(md.M * md.I * md.I, dtype=torch.float64, device="cuda")
    ctx.reconstruct(x, psi)
    torch.cuda.synchronize()
    return info, psi.cpu().numpy()


@pytest.mark.parametrize("grouped", [False, True])
def test_results_identical_alone_and_in_the_mix(lib, grouped):
    from paper_2604_23265_gb300 import rte
    meds = _mix(10, seed=1)
    srv = rte.Server(slots=4, grouped=grouped)
    ids = [srv.submit(md) for md in meds]
    got = [srv.wait(i) for i in ids]
    srv.close()
    for md, (res, psi) in zip(meds, got):
        assert res["status"] == "OK" and res["converged"], res
        info, ref = _lone(md)
        assert res["iterations"] == info["iterations"]
        np.testing.assert_array_equal(psi, ref)


@pytest.mark.parametrize("grouped", [False, True])
def test_admission_by_footprint(lib, grouped):
    from paper_2604_23265_gb300 import rte
    meds = _mix(6, seed=2)
    # a budget that holds about one request at a time: all still complete, later ones queue
    srv = rte.Server(slots=4, max_device_bytes=int(1.5 * (96 << 20)), grouped=grouped)
    ids = [srv.submit(md) for md in meds]
    res = [srv.wait(i)[0] for i in ids]
    srv.close()
    assert all(r["status"] == "OK" for r in res)
    assert max(r["queue_s"] for r in res) > 0.0
    tiny = rte.Server(slots=2, max_device_bytes=1 << 20, grouped=grouped)
    with pytest.raises(rte.RteError) as e:
        tiny.submit(meds[0])
    assert e.value.status == rte.RTE_ENOMEM
    tiny.close()


@pytest.mark.parametrize("grouped", [False, True])
def test_faults_stay_per_request(lib, grouped):
    from paper_2604_23265_gb300 import rte
    meds = _mix(5, seed=3)
    bad = W.grf_diffusive(7, I=16, M=8)
    bad.sigma_a = -bad.sigma_a                       # malformed medium
    nan = W.grf_diffusive(8, I=16, M=8)
    nan.sigma_T = nan.sigma_T.copy()
    nan.sigma_T[5] = np.nan                          # NaN medium
    srv = rte.Server(slots=3, inject_alloc_failure_id=2, grouped=grouped)
    ids = [srv.submit(meds[0]), srv.submit(meds[1]), srv.submit(bad), srv.submit(nan),
           srv.submit(meds[2]), srv.submit(meds[3])]
    res = [srv.wait(i) for i in ids]
    srv.close()
    assert res[1][0]["status"] == "ENOMEM"           # request id 2: injected failure
    assert res[2][0]["status"] == "EINVAL"
    assert res[3][0]["status"] == "EINVAL"
    for k, md in ((0, meds[0]), (4, meds[2]), (5, meds[3])):
        assert res[k][0]["status"] == "OK"
        np.testing.assert_array_equal(res[k][1], _lone(md)[1])


@pytest.mark.parametrize("grouped", [False, True])
def test_cancellation(lib, grouped):
    from paper_2604_23265_gb300 import rte
    slow = W.grf_diffusive(9, I=64, M=16, eps=1e-3)  # thousands of iterations
    quick = _mix(2, seed=4)
    srv = rte.Server(slots=2, grouped=grouped)
    i_slow = srv.submit(slow, tol=1e-12, max_iter=200000)
    i_q = [srv.submit(md) for md in quick]
    srv.cancel(i_slow)
    r_slow = srv.wait(i_slow)[0]
    rq = [srv.wait(i) for i in i_q]
    srv.close()
    assert r_slow["status"] == "ECANCELLED"
    for md, (r, psi) in zip(quick, rq):
        assert r["status"] == "OK"
        np.testing.assert_array_equal(psi, _lone(md)[1])


def _net(M, levels, seed):
    from paper_2604_23265_gb300 import rte
    shape = W.NetShape(M=M, levels=levels, c0=8, cmax=16, cc=4, ccmax=8)
    net = rte.MgNet(shape)
    net.set_params(W.init_params(shape, seed=seed, proj_scale=0.02, vcycle_scale=0.5))
    return net


@pytest.mark.parametrize("grouped", [False, True])
def test_networks_per_direction_count(lib, grouped):
    """A server holding networks for M = 8 (3 levels) and M = 16 (2 levels):
    each request with use_net runs on the network of its M when the depth fits
    its grid, else (M = 4, or I = 18 not divisible by 4 for the 3-level net)
    on block Jacobi; every result is the bits of the lone solve with the same
    preconditioner.  Two networks with one M are rejected."""
    from paper_2604_23265_gb300 import rte
    n8, n16 = _net(8, 3, 1), _net(16, 2, 2)
    assert n8.config()["M"] == 8 and n8.config()["levels"] == 3
    meds = [W.grf_diffusive(30 + i, I=I, M=M, eps=1e-2, g=0.3)
            for i, (I, M) in enumerate([(16, 8), (24, 16), (32, 8), (18, 8), (16, 4), (32, 16), (24, 8)])]
    expect_net = [True, True, True, False, False, True, True]
    srv = rte.Server(slots=3, net=[n8, n16], grouped=grouped)
    kw = dict(tol=1e-8, max_iter=400)
    ids = [srv.submit(md, use_net=True, **kw) for md in meds]
    got = [srv.wait(i) for i in ids]
    srv.close()
    for md, want, (res, psi) in zip(meds, expect_net, got):
        assert res["status"] in ("OK", "ENOTCONV"), res
        assert res["used_net"] == want
        pc = ({8: n8, 16: n16}[md.M]) if want else None
        ctx = rte.Context.from_medium(md)
        x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
        info = ctx.solve(x, pc=pc, raise_on_error=False, **kw)
        ref = torch.zeros(md.M * md.I * md.I, dtype=torch.float64, device="cuda")
        ctx.reconstruct(x, ref)
        torch.cuda.synchronize()
        assert res["iterations"] == info["iterations"] and res["fell_back"] == info["fell_back"]
        np.testing.assert_array_equal(psi, ref.cpu().numpy())
        ctx.close()
    with pytest.raises(rte.RteError):
        rte.Server(slots=1, net=[n8, _net(8, 2, 3)], grouped=grouped)
