"""Tile shapes, the autotuner and the batched persistent step.

The per-cell arithmetic of a step does not depend on how cells are grouped into tiles, so
every tile shape, and the batched kernel that steps many cases together, must reproduce the
single-case step bit for bit (the single-case paths are held to the oracle elsewhere).
The batch is the sweep of plume cases with uneven grids and conditions of the paper's
parameter study, at reduced and at full size."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2504_20742_gb300 as P
    return P


@pytest.fixture(scope="module")
def blob(P):
    from paper_2504_20742_gb300 import surrogate as S
    return S.Surrogate.load(S.default_path()).blob()


def _small_batch(n=6):
    """n cases of the sweep with their grids cut by 4 in each direction, plus a ragged one
    (grids not multiples of any tile shape)."""
    out = []
    for c, uf in cases.batch_cases(n=n):
        c = dict(c, nx=c["nx"] // 4, nr=c["nr"] // 4)
        out.append((c, np.ones(c["nr"])))
    c, _ = out[0]
    c = dict(c, nx=72, nr=20)
    out.append((c, 1.0 + 0.01 * np.sin(np.arange(20.0))))
    return out


def _single(P, c, uf, prec, nsteps, blob=None, shape=-1):
    P.ct_set_tile_shape(c, prec, shape)
    s = P.Solver(c, uf, precision=prec)
    s.init_state(0.5)
    if prec == P.CT_FP32_MLP:
        s.attach_surrogate(blob)
    s.step(nsteps, 0.5)
    d = s.diagnostics()
    P.ct_set_tile_shape(c, prec, -1)
    return s.U.clone(), d


@pytest.mark.parametrize("prec,viscous,bimodal", [(0, 0, 0), (1, 0, 0), (2, 0, 0), (0, 1, 0), (1, 1, 0),
                                                  (0, 0, 1), (1, 1, 1)])
def test_every_tile_shape_gives_the_same_state(P, blob, prec, viscous, bimodal):
    c, uf = cases.mixing_layer_case(nx=100, nr=44)
    c = dict(c, viscous=viscous, nu_t=0.05, bimodal=bimodal)
    ref, d0 = _single(P, c, uf, prec, 12, blob, 0)
    assert d0[8] == 0 and d0[7] > 0
    for shape in range(1, P.ct_tile_shape_count()):
        try:
            P.ct_set_tile_shape(c, prec, shape)
        except P.ContrailError:
            continue          # shape not built for this precision
        U, d = _single(P, c, uf, prec, 12, blob, shape)
        bits = torch.int64 if U.dtype == torch.float64 else torch.int32
        assert torch.equal(U.view(bits), ref.view(bits)), (prec, P.ct_tile_shape(shape))   # bit for bit
        assert d[0] == d0[0] and d[7] == d0[7] and d[26] == d0[26]
        # the totals are sums in another order: warp sums in the state precision, FP64 above
        tol = 1e-12 if prec == 0 else 1e-6
        for k in (1, 2, 3):
            assert abs(d[k] - d0[k]) <= tol * abs(d0[k])


def test_autotune_leaves_the_state_and_registers_a_shape(P):
    c, uf = cases.mixing_layer_case(nx=256, nr=64)
    s = P.Solver(c, uf, precision=P.CT_FP32)
    s.init_state(0.5)
    s.step(2, 0.5)
    before = s.U.clone()
    shape, ms = s.autotune(reps=3)
    torch.cuda.synchronize()
    assert torch.equal(s.U, before)
    assert 0 <= shape < P.ct_tile_shape_count() and ms[shape] > 0
    assert ms[shape] == min(m for m in ms if m > 0)
    print("tile shapes", [P.ct_tile_shape(k) for k in range(len(ms))], "ms per stage launch", ms)
    s.step(3, 0.5)
    P.ct_set_tile_shape(c, P.CT_FP32, -1)
    ref, _ = _single(P, c, uf, P.CT_FP32, 5, None, 0)
    assert torch.equal(s.U, ref)


@pytest.mark.parametrize("prec", [1, 2])
def test_batch_matches_single_case_steps(P, blob, prec):
    bc = _small_batch()
    b = P.Batch([c for c, _ in bc], [u for _, u in bc], precision=prec, blob=blob if prec == 2 else None)
    b.init_state(0.5)
    b.step(4, 0.5)
    b.step(4, 0.5)          # replays the captured graph
    db = b.diagnostics()
    assert np.all(db[:, 8] == 0)
    dts = db[:, 0]
    assert len(set(dts.tolist())) > 1          # every case keeps its own time step
    for k, (c, uf) in enumerate(bc):
        ref, d = _single(P, c, uf, prec, 8, blob)
        assert torch.equal(b.state(k), ref), k
        assert db[k, 0] == d[0] and db[k, 7] == d[7] and db[k, 27] == d[27]
        for q in (1, 2, 3):
            assert abs(db[k, q] - d[q]) <= 1e-12 * abs(d[q])


@pytest.mark.parametrize("prec", [1, 2])
def test_batched_column_sweep_matches_single_case_steps(P, blob, prec):
    """The batch through the column-sweep shape (the persistent sweep over every case's
    strips; FP32 + surrogate: then the queue kernel over every case's kept cells) against
    each case stepped alone with the default shape: bit for bit.  The mixing layer's source
    fires, so its kept cells go through the queue."""
    sweep = [k for k in range(P.ct_tile_shape_count()) if P.ct_tile_shape(k) == (28, 64)][0]
    bc = _small_batch()
    bc.append(cases.mixing_layer_case(nx=100, nr=44))   # a case whose source fires: queued cells
    b = P.Batch([c for c, _ in bc], [u for _, u in bc], precision=prec, blob=blob if prec == 2 else None)
    b.set_tile_shape(sweep)
    b.init_state(0.5)
    b.step(4, 0.5)
    b.step(4, 0.5)
    db = b.diagnostics()
    assert np.all(db[:, 8] == 0) and db[-1, 7] > 0
    for k, (c, uf) in enumerate(bc):
        ref, d = _single(P, c, uf, prec, 8, blob)
        assert torch.equal(b.state(k).view(torch.int32), ref.view(torch.int32)), k
        assert db[k, 0] == d[0] and db[k, 7] == d[7] and db[k, 26] == d[26] and db[k, 27] == d[27]
        for q in (1, 2, 3):
            assert abs(db[k, q] - d[q]) <= 1e-6 * abs(d[q])


def test_batch_shapes_autotune_and_recapture(P, blob):
    bc = _small_batch(4)
    b = P.Batch([c for c, _ in bc], [u for _, u in bc], precision=P.CT_FP32_MLP, blob=blob)
    b.init_state(0.5)
    b.step(2, 0.5)
    before = b.U.clone()
    shape, ms = b.autotune(reps=2)
    torch.cuda.synchronize()
    assert torch.equal(b.U, before)
    assert ms[shape] == min(m for m in ms if m > 0)
    b.step(3, 0.5)                      # new shape: a new graph
    after_tuned = b.U.clone()
    b.load_state(before, 0.5)
    b.set_tile_shape(0)
    b.step(1, 0.5)                      # another step count: another graph
    b.step(2, 0.5)
    assert torch.equal(b.U, after_tuned)


def test_full_size_sweep_samples(P, blob):
    """The 64-case sweep at full size (grids 256x64 .. 2048x512, about 2.5 GB of FP32 state
    in two copies) in the launch form of the benchmark; the two smallest cases are
    re-run alone and must agree bit for bit."""
    bc = cases.batch_cases(n=64)
    b = P.Batch([c for c, _ in bc], [u for _, u in bc], precision=P.CT_FP32_MLP, blob=blob)
    b.init_state(0.5)
    b.autotune(reps=1)
    b.step(3, 0.5)
    db = b.diagnostics()
    assert np.all(db[:, 8] == 0) and np.all(db[:, 27] == 3)
    sizes = [c["nx"] * c["nr"] for c, _ in bc]
    for k in np.argsort(sizes, kind="stable")[:2]:
        c, uf = bc[k]
        ref, d = _single(P, c, uf, P.CT_FP32_MLP, 3, blob)
        assert torch.equal(b.state(int(k)), ref), k
        assert db[k, 0] == d[0]
    print("active cells per case (min, max):", db[:, 7].min(), db[:, 7].max(),
          "fallbacks:", db[:, 26].sum())


def test_batch_with_optional_model_parts_matches_single_cases(P):
    """Viscous fluxes, property tables and the equilibrium model travel with each case's
    descriptor: a batch mixing them reproduces the single-case steps bit for bit (FP32)."""
    bc = _small_batch(3)
    extra = ({"viscous": 1, "nu_t": 0.2}, {"tables": 1}, {"equilibrium": 1}, {"viscous": 1, "nu_t": 0.05, "tables": 1})
    bc = [(dict(c, **e), uf) for (c, uf), e in zip(bc, extra)]
    b = P.Batch([c for c, _ in bc], [u for _, u in bc], precision=P.CT_FP32)
    b.init_state(0.5)
    b.step(5, 0.5)
    db = b.diagnostics()
    assert np.all(db[:, 8] == 0)
    for k, (c, uf) in enumerate(bc):
        ref, d = _single(P, c, uf, P.CT_FP32, 5)
        assert torch.equal(b.state(k), ref), (k, c.get("viscous"), c.get("tables"), c.get("equilibrium"))
        assert db[k, 0] == d[0]


def test_bimodal_batch_matches_single_cases(P):
    """A batch of bimodal cases (18-field states) steps each case as the single-case kernel
    does; a batch may not mix layouts."""
    bc = [(dict(c, bimodal=1), uf) for c, uf in _small_batch(3)]
    b = P.Batch([c for c, _ in bc], [u for _, u in bc], precision=P.CT_FP32)
    b.init_state(0.5)
    b.step(5, 0.5)
    db = b.diagnostics()
    assert np.all(db[:, 8] == 0)
    for k, (c, uf) in enumerate(bc):
        assert b.state(k).shape[0] == 18
        ref, d = _single(P, c, uf, P.CT_FP32, 5)
        assert torch.equal(b.state(k), ref), k
        assert db[k, 0] == d[0]
    mixed = [bc[0][0], dict(bc[1][0], bimodal=0)]
    with pytest.raises(P.ContrailError):
        P.Batch(mixed, [bc[0][1], bc[1][1]], precision=P.CT_FP32)


@pytest.mark.parametrize("make", [lambda: cases.mixing_layer_case(),
                                  lambda: (dict(cases.mixing_layer_case()[0], viscous=1, nu_t=0.05),
                                           cases.mixing_layer_case()[1]),
                                  lambda: (cases.nozzle_case(nx=400), np.ones(1))])
def test_stored_primitives_change_no_bit(P, make):
    """FP64 steps with a caller workspace keep the primitive variables of each stage's output
    for the next stage's halo; the allocation-free step converts every halo cell itself.
    Both apply the same conversion to the same state, so 20 steps agree bit for bit."""
    c, uf = make()
    a = P.Solver(c, uf, precision=P.CT_FP64)
    a.init_state(0.5)
    U0 = a.U.clone()
    a.step(20, 0.5)
    U = U0.clone()
    U1 = torch.empty_like(U)
    ufac = torch.tensor(np.asarray(uf, dtype=np.float64), device=U.device)
    P.ct_step_static(c, P.CT_FP64, ufac, U, U1, 20, 0.5)
    torch.cuda.synchronize()
    assert torch.equal(U, a.U)


def _oracle_batch():
    """Uneven cases whose phase change runs from the first step and whose trajectories are
    well conditioned (no nucleation bursts): the freezing plume on three grids and at two
    ambient temperatures, plus a cut case of the plume sweep."""
    out = []
    for nx, nr, tamb in ((96, 40, 225.0), (77, 29, 225.0), (64, 24, 215.0)):
        c, uf = cases.freezing_case(nx=nx, nr=nr)
        out.append((dict(c, T_amb=tamb), uf))
    c, _ = cases.batch_cases(n=1)[0]
    c = dict(c, nx=128, nr=32)
    out.append((c, np.ones(32)))
    return out


@pytest.mark.parametrize("prec", [1, 2])
def test_batch_cases_against_the_oracle(P, blob, prec):
    """The batched persistent kernel against the FP64 oracle itself, case by case, after 100
    steps.  FP32 transport with FP64 islands: density, momentum and energy to 1e-4 and every
    field to 5e-3 at a floor of 1e-3 of its maximum (without viscosity the vapour, the soot
    and the particle moments keep sharp contacts, where FP32 rounding moves the limiter's
    decisions: about 2e-3 there).  With the surrogate: the total liquid and ice number of
    every case within 2 % of the oracle."""
    import oracle as O
    from gpu_helpers import FLOOR_FP32, field_rel_err, report
    bc = _oracle_batch()
    b = P.Batch([c for c, _ in bc], [u for _, u in bc], precision=prec, blob=blob if prec == 2 else None)
    b.init_state(0.5)
    b.step(100, 0.5)
    db = b.diagnostics()
    assert np.all(db[:, 8] == 0)
    for k, (c, uf) in enumerate(bc):
        o = O.Oracle(c, uf)
        Uo = o.init_state()
        do = o.step(Uo, 100, 0.5)
        U = b.state(k).double().cpu().numpy()
        assert db[k, 0] == pytest.approx(do[-1, 0], rel=1e-4)      # each case its own dt
        if prec == 1:
            e = field_rel_err(U, Uo, FLOOR_FP32)
            print(f"batch case {k} ({c['nx']}x{c['nr']}), FP32 vs oracle:", report(e))
            assert np.all(e[[0, 1, 3]] <= 1e-4), report(e)
            assert np.all(e <= 5e-3), report(e)
        else:
            for f in (5, 9):
                ref = Uo[f].sum()
                if ref > 0:
                    err = abs(U[f].sum() / ref - 1.0)
                    print(f"batch case {k}, surrogate, field {f} total number vs oracle: {err:.2e}")
                    assert err <= 2e-2, (k, f, err)
