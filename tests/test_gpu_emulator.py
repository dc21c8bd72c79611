"""The emulator's CUDA kernels against the FP64 oracle (oracle.mlp,
oracle.observe).

* GEMM: every transposition, epilogue and output type, ragged shapes and
  shared operands, against float64 products of the same bf16 operands; the
  tolerance is the float32 accumulation bound K 2^-23 sum|a||b| (x2), plus
  half a bf16 ulp (2^-8 relative) when C is stored in bf16.
* Gradients of the whole ensemble (5 x 7-256x4-16) against the float64
  chain rule evaluated on the same bf16 weights and inputs.  Every GEMM
  operand (activations, back-propagated gradients) is rounded to bf16 on the
  GPU, 2^-9 relative each; over the 9 GEMMs of a layer chain the observed
  error is ~0.5%; the bound asserted is 3% of each tensor's norm and a
  cosine above 0.999.
* Adam: one and two steps against Algorithm 1 of Kingma & Ba in float64
  applied to the GPU's own gradients (float32 rounding only).
* Prediction: ensemble mean, std, output transform and fallback flags
  against numpy on the raw member outputs.
* Observations: per-cell rows and per-lattice pairs bit-exact against
  oracle.observe on the lattices read back.
"""
import numpy as np
import pytest

import cpm_workloads as cw
from oracle import mlp as omlp
from oracle import observe as oobs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2312_09317_gb300 import build as B
    B.build()
    from paper_2312_09317_gb300 import cpm
    return cpm.load()


def _bf16(x):
    """bf16 tensor on the GPU and the exact float64 values it holds."""
    t = torch.tensor(np.asarray(x), dtype=torch.float32).to(torch.bfloat16)
    return t.cuda().contiguous(), t.double().numpy()


def _p(t):
    return t.data_ptr()


GEMM_CASES = [
    # (M, N, K, batch, share_a, share_b)
    (77, 45, 39, 1, False, False),
    (128, 256, 256, 2, False, False),
    (64, 16, 7, 3, True, False),
    (5, 300, 130, 2, False, True),
    (200, 7, 300, 2, False, False),
    (16, 256, 1000, 5, False, False),
    # shapes the tensor-core (tcgen05) forward path takes when (ta, tb) = (0, 1)
    (300, 256, 256, 5, False, False),
    (129, 32, 64, 2, True, False),
    (1000, 16, 256, 3, False, False),
    (640, 128, 24, 2, False, True),
]


@pytest.mark.parametrize("ta,tb", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("case", GEMM_CASES)
@pytest.mark.parametrize("epi,c_f32", [(0, 1), (0, 0), (1, 0), (1, 1), (2, 0)])
def test_gemm_against_fp64(lib, ta, tb, case, epi, c_f32):
    M, N, K, batch, share_a, share_b = case
    rng = np.random.default_rng(M * 7 + N * 3 + K + 11 * ta + 5 * tb + epi)
    nA = 1 if share_a else batch
    nB = 1 if share_b else batch
    opA = rng.normal(0, 1, (nA, M, K))
    opB = rng.normal(0, 1, (nB, K, N))
    A_store = np.ascontiguousarray(opA.transpose(0, 2, 1) if ta else opA)
    B_store = np.ascontiguousarray(opB.transpose(0, 2, 1) if tb else opB)
    A, Ae = _bf16(A_store)
    B, Be = _bf16(B_store)
    opAe = Ae.transpose(0, 2, 1) if ta else Ae
    opBe = Be.transpose(0, 2, 1) if tb else Be
    lda = M if ta else K
    ldb = K if tb else N
    bias = torch.tensor(rng.normal(0, 1, (batch, N)), dtype=torch.float32).cuda()
    Zin = torch.tensor(rng.normal(0, 1.5, (batch, M, N)), dtype=torch.float32).cuda()
    Zout = torch.full((batch, M, N), np.nan, dtype=torch.float32).cuda()
    C = torch.zeros((batch, M, N), dtype=torch.float32 if c_f32 else torch.bfloat16).cuda()
    use_bias = epi != 2
    Z = Zin if epi == 2 else Zout
    rc = lib.cpm_mlp_gemm(ta, tb, M, N, K, batch, _p(A), lda, 0 if share_a else M * K, _p(B), ldb,
                          0 if share_b else K * N, _p(bias) if use_bias else None, N if use_bias else 0, _p(C),
                          c_f32, N, M * N, _p(Z), N, M * N, epi, None)
    assert rc == 0
    torch.cuda.synchronize()
    acc = np.einsum("bmk,bkn->bmn", np.broadcast_to(opAe, (batch, M, K)), np.broadcast_to(opBe, (batch, K, N)))
    mag = np.einsum("bmk,bkn->bmn", np.abs(np.broadcast_to(opAe, (batch, M, K))),
                    np.abs(np.broadcast_to(opBe, (batch, K, N))))
    bound = 2 * K * 2.0 ** -23 * mag + 1e-6
    b = bias.double().cpu().numpy()[:, None, :]
    if epi == 0:
        exp = acc + b
    elif epi == 1:
        z = acc + b
        exp = omlp.gelu(z)
        np.testing.assert_array_less(np.abs(Zout.double().cpu().numpy() - z), bound + 1e-6)
        bound = bound * 1.2 + 1e-6 * np.abs(exp)
    else:
        exp = acc * omlp.gelu_grad(Zin.double().cpu().numpy())
        bound = bound * 1.2 + 1e-6 * np.abs(exp)
    if not c_f32:
        bound = bound + 2.0 ** -8 * np.abs(exp)
    got = C.double().cpu().numpy()
    err = np.abs(got - exp)
    assert np.all(err <= bound), (float(err.max()), float((err / bound).max()))


@pytest.mark.parametrize("tb", [1, 0])
@pytest.mark.parametrize("epi", [1, 2])
def test_gelu_epilogue_within_the_erf_bound(lib, tb, epi):
    """The GELU (epi 1) and GELU' (epi 2) epilogues on a dense grid of bf16
    inputs in [-10, 10], against float64.  acc is made exact (one nonzero
    column of ones), so the error is the epilogue's own: erf from Abramowitz &
    Stegun 7.1.26 (|e| <= 1.5e-7) with float32 rounding and the fast
    reciprocal and exponential, bounded by 4e-7 max(1, |z|).  tb = 1 takes the
    tcgen05 forward path for epi 1, tb = 0 the mma.sync kernel."""
    grid = np.unique(torch.tensor(np.linspace(-10, 10, 6001), dtype=torch.float32)
                     .to(torch.bfloat16).double().numpy())
    M, N, K = len(grid), 16, 16
    a = np.zeros((M, K))
    a[:, 0] = grid if epi == 1 else 1.0
    A, _ = _bf16(a)
    b = np.zeros((N, K) if tb else (K, N))
    if tb:
        b[:, 0] = 1.0
    else:
        b[0, :] = 1.0
    B, _ = _bf16(b)
    bias = torch.zeros((1, N), dtype=torch.float32).cuda()
    Zin = torch.tensor(np.repeat(grid[:, None], N, axis=1), dtype=torch.float32).cuda().contiguous()
    Zout = torch.full((M, N), np.nan, dtype=torch.float32).cuda()
    C = torch.zeros((M, N), dtype=torch.float32).cuda()
    Z = Zout if epi == 1 else Zin
    rc = lib.cpm_mlp_gemm(0, tb, M, N, K, 1, _p(A), K, 0, _p(B), K if tb else N, 0,
                          _p(bias) if epi == 1 else None, 0, _p(C), 1, N, 0, _p(Z), N, 0, epi, None)
    assert rc == 0
    torch.cuda.synchronize()
    z = grid[:, None]
    exp = omlp.gelu(z) if epi == 1 else omlp.gelu_grad(z)
    got = C.double().cpu().numpy()
    err = np.abs(got - exp)
    bound = 4e-7 * np.maximum(1.0, np.abs(z))
    assert np.all(err <= bound), (float(err.max()), float(grid[np.argmax(err.max(axis=1))]))
    if epi == 1:
        np.testing.assert_array_equal(Zout.double().cpu().numpy(), np.repeat(z, N, axis=1))


SIZES = [7, 256, 256, 256, 256, 16]


def _member_params(flat, sizes, bf16_weights):
    out, o = [], 0
    for i, n in zip(sizes[:-1], sizes[1:]):
        W = flat[o:o + i * n].reshape(n, i).astype(np.float64)
        o += i * n
        b = flat[o:o + n].astype(np.float64)
        o += n
        if bf16_weights:
            W = torch.tensor(W, dtype=torch.float32).to(torch.bfloat16).double().numpy()
        out.append((W, b))
    return out


def _flat(grads):
    return np.concatenate([np.concatenate([g[0].ravel(), g[1].ravel()]) for g in grads])


@pytest.fixture(scope="module")
def net(lib):
    from paper_2312_09317_gb300 import emulator as em
    init = cw.mlp_init(3, 5, SIZES)
    e = em.Ensemble(init, 5, 7, 256, 4, 16, max_rows=1024)
    yield e, init
    e.close()


def _data(seed, rows):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (rows, 7)).astype(np.float32)
    Y = rng.normal(0, 1, (rows, 16)).astype(np.float32)
    return X, Y


def test_gradients_against_fp64_oracle(net):
    e, init = net
    e.set_params(init)
    X, Y = _data(1, 1000)
    g, loss = e.grads(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda())
    g = g.cpu().numpy()
    loss = loss.cpu().numpy()
    Xe = torch.tensor(X).to(torch.bfloat16).double().numpy()
    worst = 0.0
    for m in range(5):
        params = _member_params(init[m], SIZES, True)
        l_ref, grads, _ = omlp.loss_and_grads(params, Xe, Y)
        assert abs(loss[m] - l_ref) <= 1e-2 * l_ref, (m, loss[m], l_ref)
        o = 0
        for li, (gw, gb) in enumerate(grads):
            for ref in (gw.ravel(), gb):
                got = g[m, o:o + ref.size].astype(np.float64)
                o += ref.size
                rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
                cos = got @ ref / (np.linalg.norm(got) * np.linalg.norm(ref))
                worst = max(worst, rel)
                assert rel < 3e-2 and cos > 0.999, (m, li, rel, cos)
    print("worst relative gradient error vs fp64: %.2e" % worst)


def test_adam_steps_against_fp64(net):
    e, init = net
    e.set_params(init)
    X, Y = _data(2, 1024)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    w0 = init.astype(np.float64)
    order = torch.arange(512, dtype=torch.int32, device="cuda")
    g1, _ = e.grads(Xd, Yd, order=order, offset=0, rows=512)
    g1 = g1.cpu().numpy().astype(np.float64)
    e.train(Xd, Yd, order, 512, lr, b1, b2, eps)
    w1 = e.get_params().astype(np.float64)
    r1, m1, v1 = omlp.adam(w0, g1, 0.0, 0.0, lr, b1, b2, eps, 1)
    assert np.max(np.abs(w1 - r1)) <= 4e-7 * np.max(np.abs(w0)) + 1e-9 * lr, np.max(np.abs(w1 - r1))
    order2 = torch.arange(512, 1024, dtype=torch.int32, device="cuda")
    g2, _ = e.grads(Xd, Yd, order=order2, offset=0, rows=512)
    g2 = g2.cpu().numpy().astype(np.float64)
    e.train(Xd, Yd, order2, 512, lr, b1, b2, eps)
    w2 = e.get_params().astype(np.float64)
    r2, _, _ = omlp.adam(w1, g2, m1, v1, lr, b1, b2, eps, 2)
    assert np.max(np.abs(w2 - r2)) <= 4e-7 * np.max(np.abs(w0)) + 1e-3 * lr, np.max(np.abs(w2 - r2))


def test_training_decreases_the_loss(net):
    e, init = net
    e.set_params(init)
    rng = np.random.default_rng(5)
    X = rng.uniform(0, 1, (4096, 7)).astype(np.float32)
    Y = np.stack([np.sin(3 * X[:, i % 7]) + X[:, (i + 1) % 7] ** 2 for i in range(16)], axis=1).astype(np.float32)
    Y = (Y - Y.mean(0)) / Y.std(0)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    first = None
    for ep in range(30):
        order = torch.randperm(4096, generator=g, device="cuda").to(torch.int32)
        lt = e.train(Xd, Yd, order, 256, 2e-3, trace=True).cpu().numpy()
        if first is None:
            first = lt[0].mean()
    last = lt[-1].mean()
    assert last < 0.05 * first, (first, last)


def test_predict_against_member_outputs(net):
    e, init = net
    rng = np.random.default_rng(9)
    e.set_params(init + rng.normal(0, 0.05, init.shape).astype(np.float32))
    X = torch.from_numpy(rng.uniform(0, 1, (2500, 7)).astype(np.float32)).cuda()  # 3 chunks of 1024
    raw = e.forward(X).cpu().numpy().astype(np.float64)
    shift = rng.normal(0, 1, 16)
    scale = rng.uniform(0.5, 2, 16)
    logm = (np.arange(16) % 3 == 0).astype(np.uint8)
    sd = raw.std(axis=0)
    rmse = np.median(sd, axis=0) / 3.0
    e.set_output_transform(shift, scale, logm, rmse, 3.0)
    mean, std, fb = (t.cpu().numpy() for t in e.predict(X))
    mu = raw.mean(axis=0)
    y = mu * scale + shift
    y = np.where(logm[None] == 1, np.exp(y), y)
    np.testing.assert_allclose(mean, y, rtol=2e-5, atol=2e-5)
    np.testing.assert_allclose(std, sd, rtol=1e-4, atol=1e-5)
    ref = omlp.fallback_mask(sd, rmse, 3.0)
    tie = (np.abs(sd - 3 * rmse[None]) < 1e-4).any(axis=1)
    assert np.array_equal(fb.astype(bool)[~tie], ref[~tie])
    assert 0 < ref.sum() < len(ref)


def test_bad_row_index_is_rejected(net):
    from paper_2312_09317_gb300 import cpm
    e, init = net
    X, Y = _data(3, 64)
    order = torch.tensor([0, 5, 64, 3], dtype=torch.int32, device="cuda")
    with pytest.raises(cpm.CPMError):
        e.grads(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), order=order, offset=0, rows=4)
    g, _ = e.grads(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), order=order[:2], offset=0, rows=2)
    assert torch.isfinite(g).all()


def test_tensor_core_wait_timeout_is_reported_and_the_handle_recovers(net):
    """The failure path of the tensor-core GEMM's bounded accumulator wait:
    armed through cpm_mlp_report_next_tc_timeout, the next forward layer
    takes that path after its MMAs have completed (no GPU is stalled), the
    call returns CPM_MLP_E_CUDA with the timeout message, and the same
    handle then computes the same outputs as before the failure."""
    from paper_2312_09317_gb300 import cpm
    e, init = net
    e.set_params(init)
    X = torch.from_numpy(np.random.default_rng(11).uniform(0, 1, (700, 7)).astype(np.float32)).cuda()
    ref = e.forward(X).clone()
    assert e.lib.cpm_mlp_report_next_tc_timeout(e.h) == 0
    with pytest.raises(cpm.CPMError) as exc:
        e.forward(X)
    assert exc.value.code == -3 and "tensor-core accumulator wait timed out" in str(exc.value)
    again = e.forward(X)
    torch.cuda.synchronize()
    assert torch.equal(again, ref)
    assert e.lib.cpm_mlp_report_next_tc_timeout(None) == -1


def _observe_check(cpm, ws, n_mcs):
    b = cpm.Batch(ws)
    b.step(n_mcs)
    rows0 = b.observation_rows()
    cells = torch.empty((int(rows0[-1]), cpm.OBS_FIELDS), dtype=torch.int64, device="cuda")
    member = torch.empty((len(ws), 2), dtype=torch.int64, device="cuda")
    b.observe(cells, member)
    torch.cuda.synchronize()
    cells = cells.cpu().numpy()
    member = member.cpu().numpy()
    for k, w in enumerate(ws):
        lat = b.read_lattice(k)
        ref = oobs.cell_rows(lat, w.n_cells, w.dim)
        got = cells[rows0[k]:rows0[k + 1]]
        assert np.array_equal(got, ref), k
        assert member[k, 0] == oobs.cell_medium_pairs(lat, w.dim), k
        assert member[k, 1] == b.stats(k)["accepts"], k
    b.close()


def test_observe_2d_bit_exact(lib):
    from paper_2312_09317_gb300 import cpm
    ws = [cw.random_small(400 + k, dim=2, n=[16, 32, 48][k % 3], n_cells=3 + 2 * k, edge=3, perimeter=bool(k % 2),
                          act=bool(k % 3 == 1), obstacles=0.04 * (k % 2), a=4, c=2, P=4) for k in range(6)]
    ws += [cw.emulator_run(th, 50 + i) for i, th in enumerate(cw.sweep_points(4, 2))]
    _observe_check(cpm, ws, 5)


def test_observe_3d_bit_exact(lib):
    from paper_2312_09317_gb300 import cpm
    ws = [cw.random_small(500 + k, dim=3, n=[12, 16, 24][k % 3], n_cells=4 + k, edge=3, perimeter=True,
                          act=bool(k % 2), obstacles=0.03 * (k % 2), a=4, c=2, P=8) for k in range(4)]
    _observe_check(cpm, ws, 2)


def _observe_history(cpm, ws, burn, n_snap, every):
    b = cpm.Batch(ws)
    rows0 = b.observation_rows()
    cells = torch.empty((n_snap, int(rows0[-1]), cpm.OBS_FIELDS), dtype=torch.int64, device="cuda")
    member = torch.empty((n_snap, len(ws), 2), dtype=torch.int64, device="cuda")
    b.step(burn)
    for s in range(n_snap):
        b.observe(cells[s], member[s])
        if s + 1 < n_snap:
            b.step(every)
    out = torch.empty((len(ws), 16), dtype=torch.float64, device="cuda")
    b.summarize(cells, member, every, out)
    torch.cuda.synchronize()
    b.close()
    return rows0, cells.cpu().numpy(), member.cpu().numpy(), out.cpu().numpy()


def test_summarize_against_oracle_statistics(lib):
    """cpm_batch_summarize against oracle.observe.summary_statistics on the
    same observation history: emulator runs, then lattices of mixed sizes
    and cell counts with obstacles, perimeter and Act terms (a few cells
    vanish there, exercising the untracked-cell rules)."""
    from paper_2312_09317_gb300 import cpm
    ws = [cw.emulator_run(th, 70 + i) for i, th in enumerate(cw.sweep_points(24, 4))]
    rows0, cells, member, out = _observe_history(cpm, ws, 20, 26, 10)
    w = ws[0]
    ref = oobs.summary_statistics(cells.reshape(26, len(ws), w.n_cells + 1, 12), member, w.n_cells, (w.nx, w.ny),
                                  float(w.v_target[1]), float(w.a_target[1]), 10, w.nx * w.ny)
    assert np.isfinite(ref).all()
    np.testing.assert_allclose(out, ref, rtol=1e-9, atol=1e-12)
    ws = [cw.random_small(600 + k, dim=2, n=[16, 32, 48][k % 3], n_cells=3 + 3 * k, edge=3, perimeter=bool(k % 2),
                          act=bool(k % 3 == 1), obstacles=0.04 * (k % 2), a=4, c=2, P=4, T=[20.0, 200.0][k % 2])
          for k in range(8)]
    rows0, cells, member, out = _observe_history(cpm, ws, 3, 41, 5)
    for k, w in enumerate(ws):
        c = cells[:, rows0[k]:rows0[k + 1]][:, None]
        t1 = w.cell_type[1]
        ref = oobs.summary_statistics(c, member[:, k:k + 1], w.n_cells, (w.nx, w.ny), float(w.v_target[t1]),
                                      float(w.a_target[t1]), 5, w.nx * w.ny)
        np.testing.assert_allclose(out[k:k + 1], ref, rtol=1e-9, atol=1e-12, err_msg="lattice %d" % k)


def test_emulator_gains_over_the_cpm_alone(lib):
    """The trained ensemble against the CPM without it, at a reduced scale
    (12,288 training runs of 100 + 300 MCS): at held-out points its error
    against the mean of 16 CPM replicates is below the error of one CPM run
    on at least 10 of the 16 statistics (at this scale the smooth, low-noise
    interface and acceptance statistics are the ones it has not learnt to
    one-run precision) and by 30% on average, one point costs microseconds instead
    of a CPM run, and queries outside the training box fall back to the CPM
    far more often than queries inside it."""
    import time
    from paper_2312_09317_gb300 import emulator as em
    sim = dict(burn=100, window=300, every=10)
    X = cw.sweep_points(12288, 21)
    t0 = time.perf_counter()
    Y = em.simulate(X, np.arange(len(X)) + 10 ** 6, chunk=4096, **sim)
    t_run = (time.perf_counter() - t0) / len(X)
    emu = em.Emulator(init_seed=2, max_rows=8192)
    hist = emu.fit(X, Y, epochs=150)
    assert hist["val_rmse"].mean() < 0.35, hist["val_rmse"]
    Q, R = 32, 16
    Xq = cw.sweep_points(Q, 77)
    Yr = em.simulate(np.repeat(Xq, R, axis=0), np.arange(Q * R) + 3 * 10 ** 6, chunk=4096, **sim).reshape(Q, R, -1)
    truth = np.nanmean(Yr, axis=1)
    den = np.nanmean(np.abs(truth), axis=0)
    loo = (np.nansum(Yr, axis=1, keepdims=True) - Yr) / (R - 1)
    one_run = np.nanmean(np.abs(Yr - loo), axis=(0, 1)) / den
    Yh, _, fb = emu.predict(Xq)
    emu_err = np.nanmean(np.abs(Yh - truth), axis=0) / den
    print("emulator error", np.round(emu_err, 4), "\nsingle-run CPM error", np.round(one_run, 4))
    assert (emu_err < one_run).sum() >= 10 and emu_err.mean() < 0.7 * one_run.mean()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    emu.predict(cw.sweep_points(65536, 5))
    t_point = (time.perf_counter() - t0) / 65536
    assert t_point < 0.01 * t_run, (t_point, t_run)
    # outside the box the members disagree: a sweep there leans on the CPM
    lo = np.array([cw.SWEEP_RANGES[k][0] for k in cw.EMULATOR_PARAMS])
    hi = np.array([cw.SWEEP_RANGES[k][1] for k in cw.EMULATOR_PARAMS])
    far = lo + (hi - lo) * np.random.default_rng(4).uniform(2.0, 3.0, (512, 7))
    _, _, fb_in = emu.predict(cw.sweep_points(512, 6))
    _, _, fb_out = emu.predict(far)
    assert fb_out.mean() > 0.5 and fb_out.mean() > 5 * max(fb_in.mean(), 0.01), (fb_in.mean(), fb_out.mean())
    emu.close()
