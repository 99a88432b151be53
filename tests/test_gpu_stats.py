"""Per-cone statistics (opts.stats, scs_psd_last_stats) and the bounded
device waits.

The statistics are the error statement that comes with every result: the
eigenvalue counts behind the route, the device status and the FP64
complementarity residual <Y, Y - X> / (||Y|| ||X||) of the projection's
optimality conditions (App. D.1: the PSD cone is self-dual, so Y = Pi(X)
exactly when Y >= 0, Y - X >= 0 and <Y, Y - X> = 0).  The residual the
library reports is checked against the same quantity formed in numpy from
the returned y and the input x; the counts against the oracle's eigenvalues.

The failure test makes the one-stage reduction's group barrier run out of
its wait budget (a budget of one clock cycle): the kernel records
SCS_PSD_ETIMEOUT, returns, the cone's output is NaN, and the next call with
the default budget is correct again.  Nothing faults or hangs the GPU."""
import numpy as np
import pytest

import oracle
from paper_2606_20519_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-10
EPS = np.finfo(float).eps


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2606_20519_gb300 import _lib, build
    build.build()
    _lib.load()
    torch.cuda.init()
    return _lib


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def separated_batch(seed, sides):
    """Cones whose eigenvalues are all at least 1e-3 away from zero, so the
    counts of positive and negative eigenvalues are decided without doubt."""
    rng = W.rng_for(seed)
    svecs, lams = [], []
    for n in sides:
        if n >= 2:
            X, Q, lam = W.from_spectrum(rng, W.spectrum_vjp(rng, n, cluster=1e-3))
            svecs.append(W.to_svec(X))
            lams.append(lam)
        elif n == 1:
            v = rng.uniform(-1, 1)
            svecs.append(np.array([v]))
            lams.append(np.array([v]))
        else:
            svecs.append(np.zeros(0))
            lams.append(np.zeros(0))
    b = W.pack(svecs, sides)
    return b, lams


def check_stats(stats, b, lams, x, y, route_auto=True):
    for i, st in enumerate(stats):
        s, e = b.offsets[i], b.offsets[i + 1]
        n = int(b.sides[i])
        assert st["status"] == 0
        kp, kn = int((lams[i] > 0).sum()), int((lams[i] < 0).sum())
        assert (st["k_pos"], st["k_neg"]) == (kp, kn), i
        if n >= 2 and route_auto:
            assert st["route"] == (0 if kp <= kn else 1)
        xi, yi = x[s:e], y[s:e]
        nx, ny = np.linalg.norm(xi), np.linalg.norm(yi)
        assert abs(st["norm_x"] - nx) <= 1e-13 * max(nx, 1e-300)
        assert abs(st["norm_y"] - ny) <= 1e-13 * max(ny, 1e-300)
        if nx > 0 and ny > 0:
            c = float(yi @ (yi - xi)) / (nx * ny)
            # two FP64 sums of the same products in different orders
            slack = 2 * max(e - s, 1) * EPS * np.linalg.norm(yi - xi) / nx + 1e-300
            assert abs(st["complementarity"] - c) <= slack, (i, st["complementarity"], c)
        else:
            assert st["complementarity"] == 0.0


def test_stats_batch_fp64(lib):
    sides = [0, 1, 5, 1, 40, 90, 200, 2]
    b, lams = separated_batch(11000, sides)
    y = lib.proj_batched(dev(b.x), b.sides, opts=lib.make_opts(stats=True)).cpu().numpy()
    assert lib.status(0) == lib.OK
    stats = lib.last_stats(len(sides))
    check_stats(stats, b, lams, b.x, y)
    ref = oracle.proj_batched(b.x, b.offsets)
    assert rel(y, ref) <= TOL
    # an exact projection's residual is at rounding level
    for st in stats:
        assert abs(st["complementarity"]) <= 1e-13
    # the second call replays a recorded graph that includes the statistics
    y2 = lib.proj_batched(dev(b.x), b.sides, opts=lib.make_opts(stats=True)).cpu().numpy()
    assert lib.last_replayed(0)
    np.testing.assert_array_equal(y, y2)
    assert lib.last_stats(len(sides)) == stats


def test_stats_in_place_and_forced_routes(lib):
    sides = [120]
    b, lams = separated_batch(11100, sides)
    for side in (1, 2):
        xt = dev(b.x)
        lib.proj_batched(xt, b.sides, out=xt, opts=lib.make_opts(stats=True, side=side))
        assert lib.status(0) == lib.OK
        y = xt.cpu().numpy()
        st = lib.last_stats(1)
        check_stats(st, b, lams, b.x, y, route_auto=False)
        assert st[0]["route"] == side - 1
        assert rel(y, oracle.proj(b.x)) <= TOL


def test_stats_split_precision(lib):
    """The split path's residual, against the residual formed from its own
    output; its magnitude stays at the split path's error level."""
    n = 300
    rng = W.rng_for(11200)
    X, Q, lam = W.from_spectrum(rng, W.spectrum_precision(rng, n))
    x = W.to_svec(X)
    y = lib.proj_batched(dev(x), [n], opts=lib.make_opts(precision=lib.SPLIT_TF32, stats=True)).cpu().numpy()
    assert lib.status(0) == lib.OK
    st = lib.last_stats(1)[0]
    c = float(y @ (y - x)) / (np.linalg.norm(x) * np.linalg.norm(y))
    assert abs(st["complementarity"] - c) <= 2 * x.size * EPS
    err = rel(y, oracle.proj(x))
    assert err <= 2e-7
    assert abs(st["complementarity"]) <= 2e-7


def test_stats_vjp_and_nonfinite(lib):
    import torch
    sides = [30, 6]
    b, lams = separated_batch(11300, sides)
    g = W.rng_for(11301).standard_normal(b.x.size)
    y = torch.empty(b.x.size, dtype=torch.float64, device="cuda")
    lib.proj_vjp(dev(b.x), dev(g), b.sides, y=y, opts=lib.make_opts(stats=True))
    assert lib.status(0) == lib.OK
    check_stats(lib.last_stats(2), b, lams, b.x, y.cpu().numpy())
    x = b.x.copy()
    x[2] = np.nan
    lib.proj_batched(dev(x), b.sides, opts=lib.make_opts(stats=True))
    assert lib.status(0) == lib.ENONFINITE
    st = lib.last_stats(2)
    assert st[0]["status"] == lib.ENONFINITE and st[1]["status"] == lib.OK


def test_stats_argument_errors(lib):
    x = dev(np.ones(3))
    # statistics need an output y: the derivative alone has none
    with pytest.raises(lib.ScsPsdError):
        lib.proj_vjp(x, x, [2], opts=lib.make_opts(stats=True))
    # the count must match the last call that recorded statistics
    lib.proj_batched(x, [2], opts=lib.make_opts(stats=True))
    with pytest.raises(lib.ScsPsdError):
        lib.last_stats(2)


def test_bounded_wait_runs_out_and_recovers(lib):
    """A one-cycle budget for the spin-waits of the one-stage reduction (a
    side-300 cone is reduced by a group of many CTAs with one group barrier
    per column): the waits give up, the cone is marked SCS_PSD_ETIMEOUT and
    filled with NaN; the next call with the default budget is correct."""
    rng = W.rng_for(11400)
    n = 300
    X, Q, lam = W.from_spectrum(rng, W.spectrum_plain(rng, n))
    x = W.to_svec(X)
    xt = dev(x)
    y = lib.proj_batched(xt, [n], opts=lib.make_opts(band=1, wait_limit_cycles=1, stats=True)).cpu().numpy()
    assert lib.status(0) == lib.ETIMEOUT
    assert np.all(np.isnan(y))
    assert lib.last_stats(1)[0]["status"] == lib.ETIMEOUT
    y = lib.proj_batched(xt, [n], opts=lib.make_opts(band=1)).cpu().numpy()
    assert lib.status(0) == lib.OK
    assert rel(y, oracle.proj(x)) <= TOL
