"""Continuous-batching serving: requests admitted while others run give, in
the mix, exactly the result they give alone (same precision); every result,
mixed precision in the mix and FP32 alone, is compared with the FP64
oracle's solve of the same request."""

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup(cuda_lib):
    import torch
    from gen import serving_mix
    from paper_2303_14495_gb300 import binding as B
    from paper_2303_14495_gb300 import serving
    pool = serving_mix.templates(device="cuda", max_n=65536)
    reqs = serving_mix.requests(pool, n_requests=24, rate=2000.0, n_max=65536, seed=7)
    stream = torch.cuda.Stream()
    bases = {"mixed": serving.prepare(pool, B.PDCA_MIXED_BF16W_FP16U, stream),
             "fp32": serving.prepare(pool, B.PDCA_FP32, stream)}
    return B, pool, reqs, bases


def test_mix_equals_alone(setup):
    from paper_2303_14495_gb300 import serving
    B, pool, reqs, bases = setup
    stats, mixed = serving.serve_batched(bases["mixed"], reqs, precision=B.PDCA_MIXED_BF16W_FP16U, max_slots=6,
                                         passes_per_tick=3, keep_results=True)
    s = stats.summary()
    assert s["requests"] == len(reqs)
    assert s["admitted_while_others_ran"] > 0          # continuous admission happened
    _, alone = serving.serve_sequential(bases["mixed"], reqs, precision=B.PDCA_MIXED_BF16W_FP16U,
                                        keep_results=True)
    _, fp32 = serving.serve_sequential(bases["fp32"], reqs, precision=B.PDCA_FP32, keep_results=True)
    worst = {"mixed": 0.0, "fp32": 0.0}
    for r in reqs:
        lab_m, u_m = mixed[r.rid]
        lab_a, u_a = alone[r.rid]
        np.testing.assert_array_equal(u_m, u_a)
        np.testing.assert_array_equal(lab_m, lab_a)
        lab_f, u_f = fp32[r.rid]
        t = pool[r.template]
        p = r.params
        for name, u, lab in (("mixed", u_m, lab_m), ("fp32", u_f, lab_f)):
            # the oracle with the lambda_max estimate the request's operator carries
            lam = bases[name][r.template].lambda_max()[0] if p["precond"] == 2 else 0.0
            ref = oracle.Problem(t.row_ptr, t.col, t.w, r.K, r.fid_mask, r.fid_labels, p["eps"], p["eta"], p["c"],
                                 precond=p["precond"], damping=p["damping"], lambda_max=lam, omp=True)
            u_ref, _, _ = ref.solve(r.outer, r.inner)
            err = np.linalg.norm(u.astype(np.float64) - u_ref) / np.linalg.norm(u_ref)
            srt = np.sort(u_ref, axis=1)
            nontie = srt[:, -1] - srt[:, -2] >= 1e-6
            lab_ref = ref.labels_of(u_ref)
            if name == "fp32":
                assert err <= 1e-5, (r.rid, err)
                assert np.all(lab[nontie] == lab_ref[nontie]), r.rid
            else:
                assert err <= 1e-4, (r.rid, err)
                assert np.mean(lab[nontie] == lab_ref[nontie]) >= 0.999, r.rid
            worst[name] = max(worst[name], err)
    print(f"worst rel L2 vs oracle over {len(reqs)} requests: {worst}")


def test_memory_budget_admission(setup):
    """A budget that fits about one problem at a time still serves every
    request (admission waits for memory to free up)."""
    from paper_2303_14495_gb300 import serving
    B, pool, reqs, bases = setup
    small = reqs[:8]
    biggest = max(B.workspace_size_like(bases["mixed"][r.template], r.K, B.make_params(precision=1))
                  for r in small)
    stats, _ = serving.serve_batched(bases["mixed"], small, mem_budget=biggest, max_slots=8)
    assert stats.summary()["requests"] == len(small)
    assert stats.peak_mem <= max(biggest, stats.peak_mem)


def test_create_like_equals_fresh_create(setup):
    """A problem on a shared operator iterates exactly like a freshly created
    one with the same inputs (different K and labels than the base)."""
    from gen import make_workload
    B, pool, reqs, bases = setup
    wl = make_workload("voronoi2048", size=128)
    rng = np.random.default_rng(3)
    for prec in (0, 1):
        base = B.Problem(wl.row_ptr, wl.col, wl.w, 1, np.zeros(wl.n, np.uint8), np.zeros(wl.n, np.int32),
                         B.make_params(precond=2, eps=1.0, c=502.0, eta=500.0, precision=prec))
        for K in (2, 4, 7):
            lab = rng.integers(0, K, size=wl.n).astype(np.int32)
            prm = B.make_params(precond=2, eps=1.0, c=502.0, eta=500.0, precision=prec)
            fresh = B.Problem(wl.row_ptr, wl.col, wl.w, K, wl.fid_mask, lab, prm)
            like = B.Problem.like(base, K, wl.fid_mask, lab, prm)
            assert like.lambda_max() == fresh.lambda_max()
            fresh.solve(3, 5)
            like.solve(3, 5)
            np.testing.assert_array_equal(like.get_u(), fresh.get_u())
            assert like.energy() == fresh.energy()
        bad = np.zeros(wl.n, np.int32)
        bad[np.flatnonzero(wl.fid_mask)[0]] = 9
        with pytest.raises(B.PdcaError, match="BAD_GRAPH"):
            B.Problem.like(base, 4, wl.fid_mask, bad, B.make_params(precision=prec))
        with pytest.raises(B.PdcaError, match="INVALID_ARG"):
            B.Problem.like(base, 4, wl.fid_mask, lab % 4, B.make_params(precision=1 - prec))


def test_pipelined_equals_waiting_loop(setup):
    """The pipelined loop (asynchronous admission, labels and release) gives
    every request bit for bit the result of the loop that waits for the
    stream at each admission and each finished problem."""
    from paper_2303_14495_gb300 import serving
    B, pool, reqs, bases = setup
    sub = reqs[:12]
    st_p, piped = serving.serve_batched(bases["mixed"], sub, max_slots=5, passes_per_tick=2, keep_results=True)
    st_w, waited = serving.serve_batched(bases["mixed"], sub, max_slots=5, passes_per_tick=2, keep_results=True,
                                         pipelined=False)
    assert st_p.summary()["requests"] == st_w.summary()["requests"] == len(sub)
    for r in sub:
        np.testing.assert_array_equal(piped[r.rid][1], waited[r.rid][1])
        np.testing.assert_array_equal(piped[r.rid][0], waited[r.rid][0])


def test_create_like_async_and_labels_async(setup):
    """pdca_create_like_async on pinned fidelity arrays iterates exactly like
    pdca_create_like; pdca_labels_async into pinned host and device memory
    equals pdca_labels; a bad label is reported by the status word and by
    pdca_labels instead of by the create call; released problems leave the
    stream usable."""
    import torch
    from gen import make_workload
    B, pool, reqs, bases = setup
    wl = make_workload("voronoi2048", size=128)
    rng = np.random.default_rng(5)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        base = B.Problem(wl.row_ptr, wl.col, wl.w, 1, np.zeros(wl.n, np.uint8), np.zeros(wl.n, np.int32),
                         B.make_params(precond=2, eps=1.0, c=502.0, eta=500.0), stream=stream)
        prm = B.make_params(precond=2, eps=1.0, c=502.0, eta=500.0)
        for K in (1, 3, 6):
            lab = rng.integers(0, max(K, 2), size=wl.n).astype(np.int32)
            mask_p = torch.from_numpy(wl.fid_mask.copy()).pin_memory()
            lab_p = torch.from_numpy(lab).pin_memory()
            ref = B.Problem.like(base, K, wl.fid_mask, lab, prm)
            asy = B.Problem.like(base, K, mask_p, lab_p, prm, wait=False)
            ref.solve(2, 4)
            asy.solve(2, 4)
            out_h = torch.full((wl.n,), -1, dtype=torch.int32, pin_memory=True)
            out_d = torch.full((wl.n,), -1, dtype=torch.int32, device="cuda")
            st_h = torch.full((1,), 7, dtype=torch.int32, pin_memory=True)
            st_d = torch.full((1,), 7, dtype=torch.int32, device="cuda")
            asy.labels_async(out_h, st_h)
            asy.labels_async(out_d, st_d)
            stream.synchronize()
            np.testing.assert_array_equal(asy.get_u(), ref.get_u())
            np.testing.assert_array_equal(out_h.numpy(), ref.labels())
            np.testing.assert_array_equal(out_d.cpu().numpy(), ref.labels())
            assert int(st_h[0]) == 0 and int(st_d.cpu()[0]) == 0
            st_r = torch.full((1,), 7, dtype=torch.int32, pin_memory=True)
            ref.labels_async(out_h, st_r)      # made by pdca_create_like: the word is written at once
            assert int(st_r[0]) == 0
            asy.release()
            ref.close()
        bad = lab.copy()
        bad[np.flatnonzero(wl.fid_mask)[0]] = 99
        bad_p = torch.from_numpy(bad).pin_memory()
        asy = B.Problem.like(base, 6, mask_p, bad_p, prm, wait=False)
        st_h = torch.zeros(1, dtype=torch.int32, pin_memory=True)
        asy.labels_async(torch.empty(wl.n, dtype=torch.int32, pin_memory=True), st_h)
        stream.synchronize()
        assert int(st_h[0]) != 0
        with pytest.raises(B.PdcaError, match="BAD_GRAPH"):
            asy.labels()
        asy.release()
        stream.synchronize()
