"""The learned surrogate on the GPU against its float64 oracle (oracle/mlp.py), and the
surrogate-assisted GA: kept children are exactly decoded, runs are reproducible, and the
trained network picks better candidates than chance."""
import numpy as np
import pytest

import oracle
from oracle import mlp
import bf16_bounds as bb
from paper_1903_10741_gb300 import ffs
from paper_1903_10741_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def _setup(seed=1, N=30, g=5, batch=256):
    rng = np.random.default_rng(seed)
    prob = wl.random_instance(rng, N, g, 2, 4, 60, 5, 30, 50)
    lib_i, orc_i = ffs.Instance(prob), oracle.Instance(prob)
    gj, gs = orc_i.gene_map()
    ph, dh = mlp.gene_features(orc_i.p, orc_i.D, gj, gs)
    Y, _ = wl.random_chromosomes(rng, batch, orc_i.K, orc_i.gene_machines())
    params = mlp.init_params(orc_i.K, seed=seed)
    for k in params:
        params[k] = params[k] + rng.normal(0, 0.05, params[k].shape)
    return prob, lib_i, orc_i, ph, dh, Y, params, gs


def _p32(params):
    """The parameters as the library stores them (float32), as float64 arrays."""
    return {k: np.asarray(v, np.float32).astype(np.float64) for k, v in params.items()}


def _kpad(K):
    return (K + 127) // 128 * 128


def _worst(err, bound):
    r = err / np.maximum(bound, 1e-300)
    i = np.unravel_index(np.argmax(r), r.shape)
    return f"worst at {i}: error {err[i]:.3e}, bound {bound[i]:.3e}"


def _check_forward(sur, orc_i, Y, params):
    """Element-wise, layer by layer: each stored activation of the GPU lies in the BF16
    rounding interval of the oracle's exact sum over the GPU's own inputs to that layer,
    widened by the FP32 accumulation allowance; and every output lies within the bound
    carried through both layers from the oracle's own pass (bf16_bounds)."""
    gj, gs = orc_i.gene_map()
    p32 = _p32(params)
    ph, dh = mlp.features_f32(orc_i.p, orc_i.D, gj, gs)
    ref, c = mlp.forward_bf16(p32, Y, ph, dh, gs)
    fb = bb.forward(p32, c, _kpad(orc_i.K))
    act = sur.activations(len(Y))
    relu = lambda v: np.maximum(v, 0.0)  # noqa: E731
    # layer 1: the inputs (BF16 yh) are the oracle's; V within its float32 rounding
    lo, hi = mlp.bf16(relu(c["z1"] - fb["ez1"])), mlp.bf16(relu(c["z1"] + fb["ez1"]))
    h1 = act["h1"]
    assert np.all((lo <= h1) & (h1 <= hi)), _worst(np.abs(h1 - c["h1"]), hi - lo)
    # layer 2 on the GPU's own h1
    W2b, H = c["W2b"], c["W2b"].shape[0]
    z2 = h1 @ W2b.T + p32["b2"]
    e2 = H * bb.ACC * (np.abs(h1) @ np.abs(W2b).T) + bb.U32 * (np.abs(z2) + np.abs(p32["b2"]))
    lo, hi = mlp.bf16(relu(z2 - e2)), mlp.bf16(relu(z2 + e2))
    h2 = act["h2"]
    assert np.all((lo <= h2) & (h2 <= hi)), _worst(np.abs(h2 - mlp.bf16(relu(z2))), hi - lo)
    # output on the GPU's own h2
    o = h2 @ c["w3b"] + p32["b3"][0]
    e3 = H * bb.ACC * (np.abs(h2) @ np.abs(c["w3b"])) + 2 * bb.U32 * (np.abs(o) + abs(p32["b3"][0]))
    got = act["out"]
    assert np.all(np.abs(got - o) <= e3), _worst(np.abs(got - o), e3)
    # end to end against the oracle's own pass
    assert np.all(np.abs(got - ref) <= fb["eout"]), _worst(np.abs(got - ref), fb["eout"])
    return got, ref, fb


def test_forward_matches_oracle():
    torch = _torch()
    prob, lib_i, orc_i, ph, dh, Y, params, gs = _setup()
    sur = ffs.Surrogate(lib_i, max_batch=256)
    sur.set_params(sur.pack(params))
    got = sur.predict(torch.from_numpy(Y).cuda()).cpu().numpy().astype(np.float64)
    out, ref, fb = _check_forward(sur, orc_i, Y, params)
    assert np.array_equal(got, out)  # predict returns the outputs of that pass
    # the end-to-end bound is informative: well below the outputs' own scale
    assert np.median(fb["eout"]) < 0.2 * np.median(np.abs(ref))


def test_gradients_match_oracle():
    """Gradients element by element: the oracle's BF16-precision backward pass (exact sums)
    taken on the GPU's own stored activations, outputs and the oracle's targets, against the
    GPU's gradients, within the bound on FP32 accumulation and BF16 storage of dz2, dz1
    (bf16_bounds.backward); the masks then agree exactly."""
    torch = _torch()
    prob, lib_i, orc_i, ph, dh, Y, params, gs = _setup(seed=2)
    rng = np.random.default_rng(5)
    obj = rng.integers(10_000, 90_000, size=len(Y)).astype(np.int64)
    sur = ffs.Surrogate(lib_i, max_batch=256)
    sur.set_params(sur.pack(params))
    g, loss = sur.gradients(torch.from_numpy(Y).cuda(), torch.from_numpy(obj).cuda())
    _check_forward(sur, orc_i, Y, params)
    gj, gs = orc_i.gene_map()
    p32 = _p32(params)
    ph, dh = mlp.features_f32(orc_i.p, orc_i.D, gj, gs)
    _, c = mlp.forward_bf16(p32, Y, ph, dh, gs)
    act = sur.activations(len(Y))
    t = mlp.targets(obj)
    assert np.all(np.abs(act["t"] - t) <= bb.U32 * np.abs(t) + 1e-12)
    c["h1"], c["h2"] = act["h1"], act["h2"]
    rg, b = mlp.backward_bf16(p32, c, act["out"], t)
    z = np.zeros_like(act["h1"])
    fb = dict(ez1=z, eh1=z, ez2=z, eh2=z, eout=np.zeros(len(Y)))
    eg, info = bb.backward(p32, c, b, fb, t, _kpad(orc_i.K))
    assert not info["amb1"].any() and not info["amb2"].any()
    got = sur.unpack(g)
    for k in ("W1", "b1", "W2", "b2", "w3", "b3"):
        err = np.abs(got[k] - rg[k])
        assert np.all(err <= eg[k] + 1e-30), (k, _worst(err, eg[k]))
        # the bound is tight: typically far below the gradients themselves
        assert np.median(eg[k]) < 0.05 * np.median(np.abs(rg[k])) + 1e-12, k
    ref_loss = mlp.loss(act["out"], t)
    d = np.abs(act["out"] - t)
    assert abs(loss - ref_loss) <= 2 * np.mean(d * (bb.U32 * np.abs(t) + 1e-12)) + 2 ** -23 * ref_loss + 1e-12


def test_adam_step_is_adam():
    """The update applied by training equals one Adam step (Kingma & Ba) of the oracle
    taken with the GPU's own gradient."""
    torch = _torch()
    prob, lib_i, orc_i, ph, dh, Y, params, gs = _setup(seed=3)
    obj = np.random.default_rng(1).integers(1000, 5000, size=len(Y)).astype(np.int64)
    sur = ffs.Surrogate(lib_i, max_batch=256)
    vec = sur.pack(params)
    sur.set_params(vec)
    yd, od = torch.from_numpy(Y).cuda(), torch.from_numpy(obj).cuda()
    g, _ = sur.gradients(yd, od)
    sur.train(yd, od, lr=1e-3)
    after = sur.get_params()
    p = {"all": vec.astype(np.float64)}
    mlp.adam(p, {"all": g.astype(np.float64)}, {}, lr=1e-3)
    assert np.allclose(after, p["all"], rtol=1e-5, atol=1e-7)


def test_training_reduces_loss():
    torch = _torch()
    prob, lib_i, orc_i, ph, dh, Y, params, gs = _setup(seed=4)
    obj = np.array([orc_i.decode(y)["obj"] for y in Y], dtype=np.int64)
    sur = ffs.Surrogate(lib_i, max_batch=256, seed=9)
    yd, od = torch.from_numpy(Y).cuda(), torch.from_numpy(obj).cuda()
    first = sur.train(yd, od, lr=2e-3)
    for _ in range(60):
        last = sur.train(yd, od, lr=2e-3)
    assert last < 0.5 * first, (first, last)


def _surrogate_run(prob, gens, seed=3):
    lib_i = ffs.Instance(prob)
    pop = ffs.Population(lib_i, P=256, island=64, seed=seed)
    sur = ffs.Surrogate(lib_i, max_batch=256, seed=seed)
    pop.attach_surrogate(sur, oversample=8, lr=1e-3)
    pop.run(gens, want_schedule=False)
    return lib_i, pop, sur


def test_surrogate_ga_keeps_exact_children_and_is_reproducible():
    prob = wl.random_instance(np.random.default_rng(6), 25, 4, 2, 4, 50, 5, 30, 50)
    _, pop_a, _ = _surrogate_run(prob, 6)
    _, pop_b, _ = _surrogate_run(prob, 6)
    a, b = pop_a.read(), pop_b.read()
    for k in ("Y", "obj", "bY", "bobj"):
        assert np.array_equal(a[k], b[k]), k
    orc_i = oracle.Instance(prob)
    for i in range(0, 256, 5):
        assert a["obj"][i] == orc_i.decode(a["Y"][i])["obj"]
    # elitism: each island holds its best-ever record, and no member is better (no migration
    # happens within 6 generations, which migrate every 10)
    for i in range(len(a["bobj"])):
        assert a["bobj"][i] == orc_i.decode(a["bY"][i])["obj"]
        assert a["bobj"][i] == a["obj"][i * 64:(i + 1) * 64].min()


def test_trained_surrogate_beats_chance_on_candidates():
    """What the network adds: after the surrogate-assisted GA has run 40 generations and the
    surrogate has taken 100 more Adam steps on the final population, groups of 8 fresh
    candidates (population members with random swaps) are scored; the surrogate's pick
    beats the group's mean exact objective in more than 60 % of 256 groups.  A blind pick
    does so about half the time; 0.6 lies above its 99.9 % bound (0.5 + 3.1 / (2 sqrt 256))."""
    torch = _torch()
    prob = wl.random_instance(np.random.default_rng(8), 30, 5, 2, 4, 60, 5, 30, 50)
    lib_i, pop, sur = _surrogate_run(prob, 40, seed=5)
    d = pop.read()
    Y = d["Y"]
    yd_pop = torch.from_numpy(Y).cuda()
    od_pop = torch.from_numpy(d["obj"]).cuda()
    for _ in range(100):
        sur.train(yd_pop, od_pop, 1e-3)
    rng = np.random.default_rng(0)
    K = Y.shape[1]
    G = 256
    cands = []
    for grp in range(G):
        base = Y[rng.integers(len(Y))]
        for _ in range(8):
            y = base.copy()
            for _ in range(3):
                a, b = rng.choice(K, 2, replace=False)
                y[a], y[b] = y[b], y[a]
            cands.append(y)
    C_ = np.stack(cands).astype(np.int16)
    yd = torch.from_numpy(C_).cuda()
    score = sur.predict(yd).cpu().numpy().reshape(G, 8)
    exact = lib_i.decode(yd)["obj"].cpu().numpy().reshape(G, 8).astype(np.float64)
    picked = exact[np.arange(G), score.argmin(axis=1)]
    wins = np.mean(picked < exact.mean(axis=1))
    assert wins > 0.6, wins


def test_unscreened_surrogate_generations_equal_plain_ones():
    """Candidate 0 of every slot is the plain generation's child, so with no slot screened
    the surrogate-assisted run is the plain run, bit for bit, whatever the model says."""
    prob = wl.random_instance(np.random.default_rng(12), 22, 4, 2, 4, 50, 5, 30, 50)
    plain = ffs.Population(ffs.Instance(prob), P=256, island=64, seed=9)
    plain.run(7, want_schedule=False)
    inst = ffs.Instance(prob)
    pop = ffs.Population(inst, P=256, island=64, seed=9)
    sur = ffs.Surrogate(inst, max_batch=256, seed=3)
    pop.attach_surrogate(sur, oversample=4, lr=1e-3, train_steps=1, screen=0.0)
    pop.run(7, want_schedule=False)
    a, b = plain.read(), pop.read()
    for k in ("Y", "obj", "fit", "bY", "bobj"):
        assert np.array_equal(a[k], b[k]), k


def test_screened_slots_keep_the_best_scored_offspring():
    """With every slot screened the kept children differ from the plain run's (the model
    chooses), stay exact, and the run is reproducible."""
    prob = wl.random_instance(np.random.default_rng(13), 22, 4, 2, 4, 50, 5, 30, 50)
    runs = []
    for _ in range(2):
        inst = ffs.Instance(prob)
        pop = ffs.Population(inst, P=256, island=64, seed=9)
        sur = ffs.Surrogate(inst, max_batch=256, seed=3)
        pop.attach_surrogate(sur, oversample=4, lr=1e-3, train_steps=1, screen=1.0)
        pop.run(5, want_schedule=False)
        runs.append(pop.read())
    plain = ffs.Population(ffs.Instance(prob), P=256, island=64, seed=9)
    plain.run(5, want_schedule=False)
    assert np.array_equal(runs[0]["Y"], runs[1]["Y"])
    assert not np.array_equal(runs[0]["Y"], plain.read()["Y"])
    orc_i = oracle.Instance(prob)
    for i in range(0, 256, 9):
        assert runs[0]["obj"][i] == orc_i.decode(runs[0]["Y"][i])["obj"]


def test_forward_at_the_surrogate_workload_size():
    """The surrogate workload's instance (200 jobs, 8 stages, K = 1600, Kpad = 1664, so the
    first-layer GEMM runs with 128-wide tiles), 1024 candidates, layer by layer and element
    by element against the BF16-precision oracle."""
    torch = _torch()
    prob = wl.surrogate_large(1)
    lib_i, orc_i = ffs.Instance(prob), oracle.Instance(prob)
    rng = np.random.default_rng(3)
    Y, _ = wl.random_chromosomes(rng, 1024, orc_i.K, orc_i.gene_machines())
    params = mlp.init_params(orc_i.K, seed=3)
    for k in params:
        params[k] = params[k] + rng.normal(0, 0.02, params[k].shape)
    sur = ffs.Surrogate(lib_i, max_batch=1024)
    sur.set_params(sur.pack(params))
    got = sur.predict(torch.from_numpy(Y).cuda()).cpu().numpy().astype(np.float64)
    out, _, _ = _check_forward(sur, orc_i, Y, params)
    assert np.array_equal(got, out)


# ------------------------------------------------------------------ island keep rule

@pytest.mark.parametrize("rule", [ffs.KEEP_ISLAND, ffs.KEEP_ISLAND_OFFSPRING])
def test_island_keep_with_constant_scores_equals_plain_run(rule):
    """With every parameter zero the model scores every candidate alike, an island rule
    then keeps each slot's first candidate -- the plain generation's child -- and with no
    training the run is the plain run bit for bit (machine genes compared too)."""
    prob = wl.random_instance(np.random.default_rng(14), 22, 4, 2, 4, 50, 5, 30, 50)
    kw = dict(P=256, island=64, seed=9, mach_mode=ffs.MACH_GENE)
    plain = ffs.Population(ffs.Instance(prob), **kw)
    plain.run(7, want_schedule=False)
    inst = ffs.Instance(prob)
    pop = ffs.Population(inst, **kw)
    sur = ffs.Surrogate(inst, max_batch=256, seed=3)
    sur.set_params(np.zeros(sur.n_params, np.float32))
    pop.attach_surrogate(sur, oversample=8, lr=1e-3, train_steps=0, keep=rule)
    pop.run(7, want_schedule=False)
    a, b = plain.read(), pop.read()
    for k in ("Y", "X", "obj", "fit", "bY", "bobj"):
        assert np.array_equal(a[k], b[k]), k


def test_island_keep_ranks_each_island():
    """One generation under the island rule (8 candidates per slot, islands of 64): the
    candidates equal the oracle's offspring of the same parents bit for bit; each island
    keeps exactly its 64 best-scored rows (ties to the lower row), in row order; and every
    slot but the island's replaced one holds its kept candidate, exactly decoded."""
    prob = wl.random_instance(np.random.default_rng(15), 24, 4, 2, 4, 50, 5, 30, 50)
    P, I, F = 256, 64, 8
    inst = ffs.Instance(prob)
    pop = ffs.Population(inst, P=P, island=I, seed=11)
    sur = ffs.Surrogate(inst, max_batch=P, seed=5)
    pop.attach_surrogate(sur, oversample=F, lr=1e-3, train_steps=1, keep=ffs.KEEP_ISLAND)
    pop.run(2, want_schedule=False)
    before = pop.read()
    orc_i = oracle.Instance(prob)
    ga = oracle.GA(orc_i, P=P, island=I, seed=11)
    ga.Y[:, :ga.K], ga.X[:, :ga.K], ga.fit[:] = before["Y"], before["X"], before["fit"]
    ga.st.gen = before["gen"]
    want_Y, _, _ = ga.candidates(F)
    pop.run(1, want_schedule=False)
    c = pop.candidates(F)
    assert np.array_equal(c["Y"], want_Y)
    after = pop.read()
    for isl in range(P // I):
        rows = np.array([f * P + j for f in range(F) for j in range(isl * I, (isl + 1) * I)])
        s = c["score"][rows].astype(np.float64)
        s = np.where(np.isnan(s), np.inf, s)
        best = rows[np.lexsort((rows, s))[:I]]
        assert np.array_equal(c["keep"][isl * I:(isl + 1) * I], np.sort(best))
        held = (after["Y"][isl * I:(isl + 1) * I] == c["Y"][c["keep"][isl * I:(isl + 1) * I]]).all(axis=1)
        assert held.sum() >= I - 1
    for i in range(0, P, 7):
        assert after["obj"][i] == orc_i.decode(after["Y"][i])["obj"]


def test_exact_scores_rank_by_the_objective():
    """The diagnostic exact scoring: every candidate's score is its exact objective (the
    oracle's decode of the candidate row), so the island rule keeps the truly best rows."""
    prob = wl.random_instance(np.random.default_rng(16), 20, 4, 2, 4, 50, 5, 30, 50)
    P, I, F = 256, 64, 4
    inst = ffs.Instance(prob)
    pop = ffs.Population(inst, P=P, island=I, seed=2)
    sur = ffs.Surrogate(inst, max_batch=P, seed=2)
    sur.score_exactly(True)
    pop.attach_surrogate(sur, oversample=F, lr=1e-3, train_steps=0, keep=ffs.KEEP_ISLAND)
    pop.run(3, want_schedule=False)
    c = pop.candidates(F)
    orc_i = oracle.Instance(prob)
    for r in range(0, P * F, 13):
        assert c["score"][r] == np.float32(orc_i.decode(c["Y"][r])["obj"])
