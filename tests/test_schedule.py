"""The pair-loop and force-gather schedule the library builds for a ligand,
checked on the host without a GPU (adg_ligand_schedule): the slot and group
counts follow from the ligand, one slot is always left empty for the gather's
padding, and the modelled shared-memory wavefronts of one energy+gradient
evaluation stay close to the conflict-free count."""
import numpy as np
import pytest

from paper_2007_03678_gb300 import adg, synth as S


@pytest.fixture(scope="module")
def ff():
    from paper_2007_03678_gb300 import build
    build.build()
    return S.forcefield()


def _check(st, natoms, npairs):
    assert st["natoms"] == natoms and st["npairs"] == npairs
    assert st["nsteps"] % 2 == 0
    assert st["empty_slots"] == 32 * st["nsteps"] - npairs >= 1
    # a lane runs at most its share of the pairs, rounded up to the two-slot step
    assert st["nsteps"] <= 2 * ((npairs + 31) // 32 // 2 + 1) + 2
    assert st["pair_wavefronts"] >= st["pair_wavefronts_ideal"] > 0
    assert st["gather_wavefronts"] >= st["gather_wavefronts_ideal"]
    assert (st["gsteps"] > 0) == (npairs > 0) and (st["gather_wavefronts_ideal"] > 0) == (npairs > 0)


def test_paper_scale_ligand(ff):
    grid, rec, lig = S.workload_inputs(S.PAPER)
    st = adg.ligand_schedule(ff, lig)
    _check(st, 44, 748)
    assert st["nsteps"] == 24
    # the conflict-aware schedule: within 5 % (pair loop) and 20 % (gather,
    # after the swap search) of the conflict-free count for this ligand
    assert st["pair_wavefronts"] <= 1.05 * st["pair_wavefronts_ideal"]
    assert st["gather_wavefronts"] <= 1.20 * st["gather_wavefronts_ideal"]
    # the greedy gather alone modelled 298 wavefronts for this ligand
    assert st["gather_wavefronts"] <= 250


def test_schedule_is_deterministic(ff):
    """The gather search draws from a fixed xorshift stream and uses integer
    arithmetic only: the same ligand gets the same schedule in every call."""
    for lig in S.make_batch(8, seed=21):
        assert adg.ligand_schedule(ff, lig) == adg.ligand_schedule(ff, lig)


def test_batch_ligands(ff):
    ligs = S.make_batch(24, seed=11)
    for lig in ligs:
        st = adg.ligand_schedule(ff, lig)
        n = len(lig.type)
        assert st["natoms"] == n
        _check(st, n, st["npairs"])


def test_every_ligand_keeps_an_empty_slot(ff):
    """The gather's padding entries read an empty slot, so every schedule
    keeps one, including ligands whose pairs would fill whole two-slot steps."""
    for seed in range(200, 300):
        try:
            lig = S.make_ligand(int(10 + seed % 50), int(seed % 16), seed)
        except RuntimeError:
            continue
        st = adg.ligand_schedule(ff, lig)
        assert st["empty_slots"] >= 1, seed


def test_schedule_rejects_bad_input(ff):
    import dataclasses
    grid, rec, lig = S.workload_inputs(S.PLAIN)
    bad = dataclasses.replace(lig, type=np.full_like(lig.type, 9))
    with pytest.raises(adg.AdgError) as e:
        adg.ligand_schedule(ff, bad)
    assert e.value.code == -2  # ADG_ETYPE
    assert adg.load().adg_ligand_schedule(None, None, None) == -1  # ADG_EINVAL
