"""GPU parity: grid sort, pair lists and forces/energies/virial against the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_2006_09167_gb300 import synth
from helpers import (TOL_NET, TOL_W, all_images_within, assert_forces, canonical_pairs, check_energies,
                     rel)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_09167_gb300 import api as a
    return a


def run_forces(api, s, energy=True, virial=True, x=None):
    ctx = api.NbContext.from_system(s)
    xt = torch.tensor(s.x if x is None else x, dtype=torch.float32, device="cuda").contiguous()
    ctx.build(xt, s.box)
    f, e, w = ctx.forces(xt, energy=energy, virial=virial)
    torch.cuda.synchronize()
    assert ctx.nb_get_error() == 0
    return ctx, f.cpu().numpy(), (e.cpu().numpy() if e is not None else None), \
        (w.cpu().numpy() if w is not None else None)


def check_parity(s, ref, f, e, w, x=None, name=None):
    assert_forces(f, ref)
    if e is not None:
        check_energies(name or s.name, s, ref, e, x)
    if w is not None:
        assert np.sqrt(((w - ref["W"]) ** 2).sum() / (ref["W"] ** 2).sum()) < TOL_W
    net = np.abs(f.astype(np.float64).sum(0)).max()
    assert net < TOL_NET * np.abs(f).sum()


# ------------------------------------------------------------------- layout
def test_grid_sort_layout(api):
    s = synth.water_box(1000, 2.2 * 1.41, seed=21, rc=0.9, rlist=1.0)
    ctx = api.NbContext.from_system(s)
    xt = torch.tensor(s.x, device="cuda")
    ctx.nb_grid_sort(xt, s.box)
    perm, xq, bb = ctx.nb_debug_layout()
    st = ctx.nb_get_stats()
    real = perm[perm >= 0]
    assert np.array_equal(np.sort(real), np.arange(s.n))  # a permutation
    assert st["n_slots"] % 64 == 0
    # positions and charges are those of the permuted atoms
    assert np.array_equal(xq[perm >= 0, :3], s.x[real])
    assert np.array_equal(xq[perm >= 0, 3], s.q[real])
    # every cluster's bounding box contains its atoms
    for c in range(st["n_clusters"]):
        sl = slice(8 * c, 8 * c + 8)
        m = perm[sl] >= 0
        if not m.any():
            continue
        p = xq[sl][m, :3]
        assert np.all(p >= bb[c, 0:3]) and np.all(p <= bb[c, 4:7])
    # 2x2x2 split of each full super-cell: z halves, then y halves, then x halves
    for si in range(st["n_superclusters"]):
        sl = slice(64 * si, 64 * si + 64)
        if np.any(perm[sl] < 0):
            continue
        p = xq[sl, :3]
        assert p[:32, 2].max() <= p[32:, 2].min()
        for h in range(2):
            q = p[32 * h:32 * h + 32]
            assert q[:16, 1].max() <= q[16:, 1].min()
            for g in range(2):
                r = q[16 * g:16 * g + 16]
                assert r[:8, 0].max() <= r[8:, 0].min()
    # columns: super-cells of a column are ordered by z
    # (consecutive super-cells in a column share x/y column bounds)
    del xt


# --------------------------------------------------------------- coverage
@pytest.mark.parametrize("which", ["outer", "inner"])
def test_pairlist_covers_plain_definition(api, which):
    s = synth.water_648()  # rlist 1.0 > L/2: several images per pair in the outer list
    ctx = api.NbContext.from_system(s)
    xt = torch.tensor(s.x, device="cuda")
    ctx.build(xt, s.box)
    if which == "outer":
        got = canonical_pairs(ctx.nb_debug_export_pairs(api.NB_LIST_OUTER))
        want = all_images_within(s.x, s.box, s.rlist, s.excl_off, s.excl_idx)
    else:
        got = canonical_pairs(ctx.nb_debug_export_pairs(api.NB_LIST_INNER))
        want = {tuple(int(v) for v in r) for r in canonical_pairs(oracle.pairs_within(s, s.r_in))}
    assert len(got) == len(set(got)), "duplicate image pairs in the list"
    missing = want - set(got)
    assert not missing, f"{len(missing)} pairs missing, e.g. {sorted(missing)[:5]}"
    # nothing excluded is listed
    ex = {(i, int(j)) for i in range(s.n) for j in s.excl_idx[s.excl_off[i]:s.excl_off[i + 1]]}
    assert not any((g[0], g[1]) in ex for g in got)


def test_pairlist_coverage_polymer_like_exclusions(api):
    # random chains with 1-2/1-3 exclusions across clusters, Ewald, several tiles
    s = synth.polymer_water_box(seed=5, n_chain=6, chain_len=40, n_water=1400, box_len=3.6,
                                water_side=12, rc=1.0, rlist=1.1)
    ctx = api.NbContext.from_system(s)
    xt = torch.tensor(s.x, device="cuda")
    ctx.build(xt, s.box)
    got = canonical_pairs(ctx.nb_debug_export_pairs(api.NB_LIST_INNER))
    want = {tuple(int(v) for v in r) for r in canonical_pairs(oracle.pairs_within(s, s.r_in))}
    assert len(got) == len(set(got))
    assert not (want - set(got))
    ex = {(i, int(j)) for i in range(s.n) for j in s.excl_idx[s.excl_off[i]:s.excl_off[i + 1]]}
    assert not any((g[0], g[1]) in ex for g in got)


def test_search_segments_same_pairs(api):
    """The pair search's column segments change the work items, not the pair set:
    outer and inner lists export the same image pairs for 1, 3 and 8 segments as
    for the library's choice, and the forces agree."""
    s = synth.polymer_water_box(seed=6, n_chain=4, chain_len=40, n_water=1200, box_len=3.4,
                                water_side=11, rc=1.0, rlist=1.1)
    xt = torch.tensor(s.x, device="cuda")
    ref = None
    for seg in (0, 1, 3, 8):
        ctx = api.NbContext.from_system(s)
        ctx.nb_set_search_segments(seg)
        ctx.build(xt, s.box)
        outer = canonical_pairs(ctx.nb_debug_export_pairs(api.NB_LIST_OUTER))
        inner = canonical_pairs(ctx.nb_debug_export_pairs(api.NB_LIST_INNER))
        f, e, _ = ctx.forces(xt, energy=True)
        torch.cuda.synchronize()
        got = (set(outer), set(inner), f.cpu().numpy(), e.cpu().numpy())
        assert len(outer) == len(got[0]) and len(inner) == len(got[1])
        if ref is None:
            ref = got
            continue
        assert got[0] == ref[0] and got[1] == ref[1], f"segments {seg}: different pair set"
        assert_forces(got[2], ref[2], tol_rms=1e-6, tol_atom=1e-5)
        # other items sum the per-lane FP32 energy terms in another order: the totals agree to
        # the FP32 summation error (amplified by the Coulomb sum's cancellation), within 1e-6
        assert rel(got[3][0], ref[3][0]) < 1e-6 and rel(got[3][1], ref[3][1]) < 1e-6
        assert ctx.nb_get_error() == 0
    ctx = api.NbContext.from_system(s)
    for bad in (-1, 9):
        with pytest.raises(api.NbError):
            ctx.nb_set_search_segments(bad)


# ----------------------------------------------------------------- forces
def test_forces_648_reaction_field(api):
    s = synth.water_648()
    _, f, e, w = run_forces(api, s)
    ref = oracle.brute(s)
    check_parity(s, ref, f, e, w, name="648 water, reaction field")


def test_forces_24k_six_types(api):
    # the differentiation box's forward evaluation (Ewald, six LJ types)
    s = synth.water_24k_types()
    _, f, e, w = run_forces(api, s)
    ref = oracle.celllist(s)
    check_parity(s, ref, f, e, w, name="24k water, 6 LJ types, Ewald")


@pytest.mark.parametrize("n_mol,box_len", [(1000, 3.1), (3375, 4.66)])
def test_forces_water_ewald_small(api, n_mol, box_len):
    s = synth.water_box(n_mol, box_len, seed=31 + n_mol, rc=1.0, rlist=1.1)
    _, f, e, w = run_forces(api, s)
    ref = oracle.celllist(s)
    check_parity(s, ref, f, e, w)


def test_forces_flags_agree(api):
    s = synth.water_box(1000, 3.1, seed=41, rc=1.0, rlist=1.1)
    ctx = api.NbContext.from_system(s)
    xt = torch.tensor(s.x, device="cuda")
    ctx.build(xt, s.box)
    outs = [ctx.forces(xt, energy=en, virial=vi) for en in (False, True) for vi in (False, True)]
    torch.cuda.synchronize()
    f0 = outs[0][0].cpu().numpy()
    for f, e, w in outs[1:]:
        assert_forces(f.cpu().numpy(), f0, tol_rms=1e-6, tol_atom=1e-5)
    assert outs[1][2] is not None and outs[2][1] is not None


def test_forces_out_of_box_images(api):
    # caller coordinates shifted by whole box vectors give the same physics
    s = synth.water_box(1000, 3.1, seed=43, rc=1.0, rlist=1.1)
    rng = np.random.default_rng(0)
    shift = rng.integers(-2, 3, size=(s.n, 3)) * s.box
    x2 = (s.x.astype(np.float64) + shift).astype(np.float32)
    _, f, e, w = run_forces(api, s, x=x2)
    ref = oracle.celllist(s, x=x2)
    check_parity(s, ref, f, e, w, x=x2)


def test_forces_polymer_water_small(api):
    s = synth.polymer_water_box(seed=6, n_chain=8, chain_len=50, n_water=2400, box_len=4.3,
                                water_side=14, rc=1.2, rlist=1.3)
    _, f, e, w = run_forces(api, s)
    ref = oracle.celllist(s)
    check_parity(s, ref, f, e, w)


def test_forces_96k_full_size_sampled(api):
    s = synth.water_96k()
    _, f, e, w = run_forces(api, s)
    rng = np.random.default_rng(3)
    sub = np.sort(rng.choice(s.n, 4000, replace=False))
    ref = oracle.celllist(s, subset=sub)
    assert_forces(f[sub], ref)
    full = oracle.celllist(s)
    check_energies("96k water, Ewald", s, full, e)
    assert np.sqrt(((w - full["W"]) ** 2).sum() / (full["W"] ** 2).sum()) < TOL_W
    assert_forces(f, full)


def test_count_pairs_matches_oracle(api):
    s = synth.water_box(1000, 3.1, seed=45, rc=1.0, rlist=1.1)
    ctx, f, e, w = run_forces(api, s)
    within, evald = ctx.nb_count_pairs()
    assert within == oracle.brute(s)["npairs"]
    assert evald >= within and evald % 64 == 0


def test_forces_1p5M_polymer_water_full_size(api):
    # the full heterogeneous 1.5M-atom box: sampled forces, full energies and virial
    s = synth.polymer_water_box()
    ctx, f, e, w = run_forces(api, s)
    st = ctx.nb_get_stats()
    assert st["n_atoms"] == 1_500_000
    rng = np.random.default_rng(5)
    # chain atoms (the first 225,000) and waters both sampled
    sub = np.sort(np.concatenate([rng.choice(225000, 1500, replace=False),
                                  225000 + rng.choice(s.n - 225000, 1500, replace=False)]))
    ref = oracle.celllist(s, subset=sub)
    assert_forces(f[sub], ref)
    full = oracle.celllist(s)
    check_energies("1.5M polymer + water, Ewald", s, full, e)
    assert np.sqrt(((w - full["W"]) ** 2).sum() / (full["W"] ** 2).sum()) < TOL_W
    assert_forces(f, full)
    net = np.abs(f.astype(np.float64).sum(0)).max()
    assert net < TOL_NET * np.abs(f).sum()


@pytest.mark.parametrize("n", [1000, 20000])
def test_forces_argon_lj_only(api, n):
    # LJ argon (no charges, Lennard-Jones-only kernel flavour) at the paper's density
    s = synth.argon_box(n, seed=13, rc=1.1, rlist=1.2)
    _, f, e, w = run_forces(api, s)
    ref = oracle.celllist(s)
    check_parity(s, ref, f, e, w)
    assert e[1] == 0.0
