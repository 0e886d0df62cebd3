"""Search server: requests served concurrently in run slices must give exactly
the result of the same search run alone (and the oracle's), whatever else
is in flight; the device-memory budget makes requests queue; cancel, poll
and wait time-outs behave as include/xyz.h states.
"""
import threading

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xyz():
    from paper_1610_05108_gb300 import build, xyz as mod
    build.build()
    mod.load()
    return mod


def _data(n, p, seed, planted=((0, 1),), flip=0.1):
    rng = np.random.default_rng(seed)
    X = np.asfortranarray((rng.integers(0, 2, size=(n, p), dtype=np.int8) * 2 - 1).astype(np.int8))
    Ys = []
    for a, c in planted:
        y = (X[:, a] * X[:, c]).astype(np.int8)
        f = rng.random(n) < flip
        y[f] = -y[f]
        Ys.append(y)
    return X, Ys


def _arr(res):
    if len(res) == 0:
        return np.zeros((0, 3), np.int32)
    return np.stack([res["j"], res["k"], res["agree"]], axis=1).astype(np.int32)


def test_served_equals_alone_and_oracle(xyz, orc):
    XA, YA = _data(200, 2500, 1, planted=((3, 7), (10, 900), (5, 6)))
    XB, YB = _data(131, 1700, 2, planted=((0, 1), (44, 1600)))
    jobs = [  # (dataset, Y index or None, L, M, kappa, seed)
        (0, None, 60, 9, 0.3, 11), (0, 1, 45, 8, 0.25, 12), (1, None, 70, 9, 0.2, 13),
        (0, 2, 33, 10, 0.3, 14), (1, 1, 51, 7, 0.3, 15), (0, None, 64, 30, 0.1, 16),
        (1, None, 40, 33, 0.0, 17), (0, 0, 1, 9, 0.3, 18),
    ]
    data = [(XA, YA), (XB, YB)]
    with xyz.Server(workers=3, hbm_budget_bytes=8 << 30, slice_runs=7) as srv:
        ds = [srv.add_dataset(X, Ys[0]) for X, Ys in data]
        reqs = []
        for d, yi, L, M, kappa, seed in jobs:
            Y = None if yi is None else data[d][1][yi]
            reqs.append(srv.submit(ds[d], L, M, kappa, seed, Y=Y))
        results = [srv.wait(r, timeout_ms=120000) for r in reqs]
        st = srv.stats()
    assert st["completed"] == len(jobs) and st["failed"] == 0 and st["canceled"] == 0
    assert st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"]
    for (d, yi, L, M, kappa, seed), (got, lat) in zip(jobs, results):
        X, Ys = data[d]
        Y = Ys[0] if yi is None else Ys[yi]
        with xyz.create(X, Y) as ctx:
            alone = ctx.search(L, M, kappa, seed)
        assert np.array_equal(got, alone), (d, yi, L, M)
        assert lat > 0
        if M <= 10:
            assert np.array_equal(_arr(got), orc.xyz(X, Y, L, M, kappa, seed)), (d, yi, L, M)
    assert sum(len(r[0]) for r in results) > 0


def test_concurrent_submitters(xyz):
    X, Ys = _data(180, 2000, 3, planted=((1, 2), (3, 4), (5, 6), (7, 8)))
    with xyz.Server(workers=2, hbm_budget_bytes=8 << 30, slice_runs=5) as srv:
        d = srv.add_dataset(X, Ys[0])
        out = {}

        def client(i):
            r = srv.submit(d, 30 + i, 9, 0.3, 100 + i, Y=Ys[i % len(Ys)])
            out[i] = srv.wait(r, timeout_ms=120000)[0]

        th = [threading.Thread(target=client, args=(i,)) for i in range(6)]
        for t in th:
            t.start()
        for t in th:
            t.join(timeout=300)
        assert len(out) == 6
    with xyz.create(X, Ys[0]) as ctx:
        for i in range(6):
            ctx.set_y(Ys[i % len(Ys)])
            assert np.array_equal(out[i], ctx.search(30 + i, 9, 0.3, 100 + i)), i


def test_budget_makes_requests_queue(xyz):
    X, Ys = _data(160, 3000, 4)
    with xyz.Server(workers=2, hbm_budget_bytes=8 << 30, slice_runs=4) as probe:
        probe.add_dataset(X, Ys[0])
        packed = probe.stats()["device_bytes"]
    # room for the dataset only: one request at a time may be admitted
    with xyz.Server(workers=2, hbm_budget_bytes=packed + 1, slice_runs=4) as srv:
        d = srv.add_dataset(X, Ys[0])
        reqs = [srv.submit(d, 40, 9, 0.3, 200 + i) for i in range(4)]
        st = srv.stats()
        assert st["queued"] + st["active"] + st["completed"] == 4
        assert st["queued"] >= 2 or st["completed"] >= 2
        got = [srv.wait(r, timeout_ms=120000)[0] for r in reqs]
        st = srv.stats()
        assert st["completed"] == 4 and st["queued"] == 0 and st["active"] == 0
    with xyz.create(X, Ys[0]) as ctx:
        for i in range(4):
            assert np.array_equal(got[i], ctx.search(40, 9, 0.3, 200 + i))


def test_reservation_sized_from_workspace(xyz):
    # a request's reservation is its share of the workers' workspace growth,
    # sized by the library's workspace rules at admission: on fresh workers
    # it is of the order of what they measure after serving it
    X, Ys = _data(160, 3000, 5)
    with xyz.Server(workers=2, hbm_budget_bytes=8 << 30, slice_runs=64) as srv:
        d = srv.add_dataset(X, Ys[0])
        base = srv.stats()["device_bytes"]
        r = srv.submit(d, 2000, 9, 0.3, 7)
        held = srv.stats()["device_bytes"] - base       # reservation (+ any workspace measured already)
        got = srv.wait(r, timeout_ms=120000)[0]
        after = srv.stats()["device_bytes"] - base      # the workers' measured workspaces
    assert after > 0
    assert held >= 0.5 * after
    with xyz.create(X, Ys[0]) as ctx:
        assert np.array_equal(got, ctx.search(2000, 9, 0.3, 7))


def test_cancel_timeout_poll(xyz):
    X, Ys = _data(150, 4000, 5)
    with xyz.Server(workers=1, hbm_budget_bytes=8 << 30, slice_runs=16) as srv:
        d = srv.add_dataset(X, Ys[0])
        long_req = srv.submit(d, 200000, 9, 0.3, 1)
        with pytest.raises(xyz.XyzError) as e:
            srv.wait(long_req, timeout_ms=0)
        assert e.value.code == xyz.XYZ_ETIMEDOUT
        with pytest.raises(xyz.XyzError) as e:
            srv.poll(long_req)
        assert e.value.code == xyz.XYZ_EAGAIN
        queued = srv.submit(d, 10, 9, 0.3, 2)
        srv.cancel(long_req)
        with pytest.raises(xyz.XyzError) as e:
            srv.wait(long_req, timeout_ms=60000)
        assert e.value.code == xyz.XYZ_ECANCELED
        got, lat = srv.wait(queued, timeout_ms=60000)
        with xyz.create(X, Ys[0]) as ctx:
            assert np.array_equal(got, ctx.search(10, 9, 0.3, 2))
        st = srv.stats()
        assert st["canceled"] == 1 and st["completed"] == 1
        # a retired request is unknown afterwards
        with pytest.raises(xyz.XyzError) as e:
            srv.poll(queued)
        assert e.value.code == xyz.XYZ_EINVAL


def test_server_argument_errors(xyz):
    X, Ys = _data(64, 100, 6)
    with pytest.raises(xyz.XyzError) as e:
        xyz.Server(workers=0)
    assert e.value.code == xyz.XYZ_EINVAL
    with xyz.Server(workers=1, hbm_budget_bytes=1024, slice_runs=4) as srv:
        with pytest.raises(xyz.XyzError) as e:
            srv.add_dataset(X, Ys[0])
        assert e.value.code == xyz.XYZ_ENOMEM
    with xyz.Server(workers=1, hbm_budget_bytes=1 << 30, slice_runs=4) as srv:
        d = srv.add_dataset(X, Ys[0])
        for args in ((d + 1, 5, 5, 0.3, 0), (d, 0, 5, 0.3, 0), (d, 5, 65, 0.3, 0), (d, 5, 5, 1.5, 0)):
            with pytest.raises(xyz.XyzError) as e:
                srv.submit(*args)
            assert e.value.code == xyz.XYZ_EINVAL
        bad = Ys[0].copy()
        bad[3] = 0
        with pytest.raises(xyz.XyzError) as e:
            srv.submit(d, 5, 5, 0.3, 0, Y=bad)
        assert e.value.code == xyz.XYZ_EINVAL
        r = srv.submit(d, 5, 5, 0.3, 0)
        got, _ = srv.wait(r, timeout_ms=60000)
        with xyz.create(X, Ys[0]) as ctx:
            assert np.array_equal(got, ctx.search(5, 5, 0.3, 0))
