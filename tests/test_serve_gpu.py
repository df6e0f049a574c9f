"""Serving (hs_submit / hs_poll): continuous batching on one plan.

* each request's H, S are bitwise identical alone (hs_assemble) and in a mix
  of concurrently running requests of uneven N_G;
* admission never exceeds the HBM budget (every request reports the admitted
  footprint at its admission) and all requests still complete in a tight budget;
* a served request matches the CPU oracle;
* host-side errors: over-budget -> HS_ENOMEM, bad arguments / unknown ticket ->
  HS_EINVAL, hs_set_t while requests are in flight -> HS_EBUSY, short polls ->
  HS_PENDING / HS_ETIMEDOUT.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import assemble, rel_frobenius  # noqa: E402
from paper_1611_00606_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def hs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_00606_gb300 import hs as _hs
    return _hs


@pytest.fixture(scope="module")
def pool():
    """A pool of coefficients (N_A=6, N_L=25, up to 640 columns) and shared T, U."""
    w = synth.Workload("pool", 6, 25, 640, (2,), seed=31)
    return w, synth.make_inputs(w)


def _dev_T(hs, d):
    return [hs.to_device_T(d[k]) for k in ("T_AA", "T_AB", "T_BB")], hs.to_device_U(d["U"])


@pytest.mark.parametrize("precision", ["split_bf16", "fp64"])
def test_alone_equals_mix(hs, pool, precision):
    w, d = pool
    A, B = hs.to_device_coef(d["A"]), hs.to_device_coef(d["B"])
    T, U = _dev_T(hs, d)
    sizes = [640, 37, 257, 500, 129, 1, 400, 640]
    with hs.Plan(w.N_A, w.N_L, w.N_G, precision) as p:
        alone = []
        for n in sizes:
            H, S, _ = hs.hs_assemble(p.h, A[:, :n], B[:, :n], *T, U, w.N_A, w.N_L, n)
            alone.append((H.clone(), S.clone()))
        outs = [(hs.empty_hs(n), hs.empty_hs(n)) for n in sizes]
        tickets = [hs.hs_submit(p.h, A, B, U, n, H, S) for n, (H, S) in zip(sizes, outs)]
        for t in tickets:
            rc, info = hs.hs_poll(p.h, t, -1)
            assert rc == hs.HS_OK and info["ms_latency"] >= info["ms_queue"] >= 0
    torch.cuda.synchronize()
    for (Ha, Sa), (Hm, Sm) in zip(alone, outs):
        assert torch.equal(Ha, Hm) and torch.equal(Sa, Sm)


def test_admission_respects_budget(hs, pool):
    w, d = pool
    A, B = hs.to_device_coef(d["A"]), hs.to_device_coef(d["B"])
    T, U = _dev_T(hs, d)
    with hs.Plan(w.N_A, w.N_L, w.N_G, "split_bf16") as p0:
        hs.hs_set_t(p0.h, *T)
        fp_max = hs.hs_footprint(p0.h, w.N_G)
    budget = int(2.5 * fp_max)  # at most two of the widest requests at once
    sizes = [640, 640, 640, 300, 640, 100, 640, 640]
    with hs.Plan(w.N_A, w.N_L, w.N_G, "split_bf16", 0, budget) as p:
        hs.hs_set_t(p.h, *T)
        outs = [(hs.empty_hs(n), hs.empty_hs(n)) for n in sizes]
        tickets = [hs.hs_submit(p.h, A, B, U, n, H, S) for n, (H, S) in zip(sizes, outs)]
        # the cached factor is in use: refactoring while requests run is refused
        try:
            hs.hs_set_t(p.h, *T)
        except hs.HSError as e:
            assert e.code == hs.HS_EBUSY
        infos = []
        for t in tickets:
            rc, info = hs.hs_poll(p.h, t, -1)
            assert rc == hs.HS_OK
            infos.append(info)
        assert all(i["inflight_bytes"] <= budget for i in infos)
        assert max(i["inflight_bytes"] for i in infos) > fp_max  # requests did overlap
        with hs.Plan(w.N_A, w.N_L, w.N_G, "split_bf16") as ref:
            for n, (H, S) in zip(sizes, outs):
                Hr, Sr, _ = hs.hs_assemble(ref.h, A[:, :n], B[:, :n], *T, U, w.N_A, w.N_L, n)
                assert torch.equal(Hr, H) and torch.equal(Sr, S)


def test_served_request_matches_oracle(hs, pool):
    w, d = pool
    n = 333
    A, B = hs.to_device_coef(d["A"]), hs.to_device_coef(d["B"])
    T, U = _dev_T(hs, d)
    with hs.Plan(w.N_A, w.N_L, w.N_G, "split_bf16") as p:
        hs.hs_set_t(p.h, *T)
        H, S = hs.empty_hs(n), hs.empty_hs(n)
        t = hs.hs_submit(p.h, A, B, U, n, H, S)
        rc, info = hs.hs_poll(p.h, t, -1)
        assert rc == hs.HS_OK and info["n_fallback"] == 1
    Hr, Sr = assemble(d["A"][:, :n], d["B"][:, :n], d["T_AA"], d["T_AB"], d["T_BB"], d["U"],
                      w.N_A, w.N_L)
    assert rel_frobenius(H.cpu().numpy(), Hr) <= 1e-10
    assert rel_frobenius(S.cpu().numpy(), Sr) <= 1e-10


def test_serving_errors(hs, pool):
    w, d = pool
    A, B = hs.to_device_coef(d["A"]), hs.to_device_coef(d["B"])
    T, U = _dev_T(hs, d)
    H, S = hs.empty_hs(w.N_G), hs.empty_hs(w.N_G)
    with hs.Plan(w.N_A, w.N_L, w.N_G, "split_bf16") as p0:
        hs.hs_set_t(p0.h, *T)
        fp = hs.hs_footprint(p0.h, w.N_G)
    with hs.Plan(w.N_A, w.N_L, w.N_G, "split_bf16", 0, fp - 1) as p:
        # no factor yet
        with pytest.raises(hs.HSError) as e:
            hs.hs_submit(p.h, A, B, U, w.N_G, H, S)
        assert e.value.code == hs.HS_EINVAL
        hs.hs_set_t(p.h, *T)
        # budget one byte short of the widest request: it can never be admitted
        with pytest.raises(hs.HSError) as e:
            hs.hs_submit(p.h, A, B, U, w.N_G, H, S)
        assert e.value.code == hs.HS_ENOMEM
        with pytest.raises(hs.HSError) as e:
            hs.hs_submit(p.h, A, B, U, w.N_G + 1, hs.empty_hs(w.N_G + 1), hs.empty_hs(w.N_G + 1))
        assert e.value.code == hs.HS_EINVAL
        with pytest.raises(hs.HSError) as e:
            hs.hs_poll(p.h, 12345, 0)
        assert e.value.code == hs.HS_EINVAL
    big = synth.Workload("big", 40, 121, 2048, (), seed=32)
    db = synth.make_inputs(big)
    Ab, Bb = hs.to_device_coef(db["A"]), hs.to_device_coef(db["B"])
    Tb, Ub = _dev_T(hs, db)
    Hb, Sb = hs.empty_hs(big.N_G), hs.empty_hs(big.N_G)
    with hs.Plan(big.N_A, big.N_L, big.N_G, "split_bf16") as p:
        hs.hs_set_t(p.h, *Tb)
        t = hs.hs_submit(p.h, Ab, Bb, Ub, big.N_G, Hb, Sb)
        rc, _ = hs.hs_poll(p.h, t, 0)
        assert rc in (hs.HS_PENDING, hs.HS_OK)
        if rc == hs.HS_PENDING:
            rc, _ = hs.hs_poll(p.h, t, 1)
            assert rc in (hs.HS_ETIMEDOUT, hs.HS_OK)
            if rc == hs.HS_ETIMEDOUT:
                rc, _ = hs.hs_poll(p.h, t, -1)
        assert rc == hs.HS_OK
