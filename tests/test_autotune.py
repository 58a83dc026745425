"""Host logic of the autotuner (no GPU): candidate sets, classes, the choice
of the fastest candidate, skipped candidates, and the JSON round trip."""
import pytest

from paper_2506_02130_gb300 import autotune as AT, fv, workloads as W


def test_candidates_respect_the_mixed_sigma_floor():
    mixed = AT.candidates(fv.FV_MIXED, ("auto", "type3"))
    fp64 = AT.candidates(fv.FV_FP64, ("auto", "type3"))
    assert {c.transform for c in AT.candidates(fv.FV_MIXED)} == {"auto"}
    assert {c.upsampfac for c in mixed} == {1.5, 2.0}
    assert {c.upsampfac for c in fp64} == {1.25, 2.0}
    for cs, n in ((mixed, 16), (fp64, 16)):
        assert {c.spread for c in cs} == {"gather", "scatter"}
        assert {c.fft_max_radix for c in cs} == {8, 16}
        assert {c.transform for c in cs} == {"auto", "type3"}
        assert len(set(cs)) == n


def test_class_key_groups_by_precision_array_and_octave():
    k = AT.class_key
    assert k(fv.FV_MIXED, 37, 1024) == k(fv.FV_MIXED, 37, 2047)
    assert k(fv.FV_MIXED, 37, 1023) != k(fv.FV_MIXED, 37, 1024)
    assert k(fv.FV_MIXED, 37, 1500) != k(fv.FV_FP64, 37, 1500)
    assert k(fv.FV_MIXED, 37, 1500) != k(fv.FV_MIXED, 61, 1500)


def _slices():
    return W.config_batch(seed=5, n_slices=40, radii=(3, 4), n_src_range=(1000, 4000))


def test_tuner_takes_the_fastest_candidate_per_class(tmp_path):
    calls = []

    def timer(choice, bs):
        calls.append((choice, AT.key_of(bs)))
        if choice.upsampfac == 1.25:
            raise fv.FvError(fv.FV_ERR_UNSUPPORTED, "grid too large")
        # fastest: sigma 2, scatter, radix 8 for fp64; sigma 1.5, gather, radix 16 for mixed
        best = AT.Choice(2.0, "scatter", 8) if AT.precision_of(bs) == fv.FV_FP64 else AT.Choice(1.5, "gather", 16)
        return 1.0 if choice == best else 2.0 + choice.fft_max_radix / 100

    slices = _slices()
    t = AT.Autotuner(timer, routes=("auto", "type3"))
    table = t.tune(slices, AT.key_of, AT.precision_of)
    keys = {AT.key_of(s) for s in slices}
    assert set(table) == keys
    # one representative per class, every candidate tried once on it (no bin round: the winners are not
    # type-3 gather plans)
    assert len(calls) == 16 * len(keys)
    for s in slices:
        c = t.choice(AT.precision_of(s), len(s.problem.ant_enu), s.problem.sky.n_src)
        assert c == (AT.Choice(2.0, "scatter", 8) if s.precision == "fp64" else AT.Choice(1.5, "gather", 16))
    # tuned classes are not timed again
    n = len(calls)
    t.tune(slices, AT.key_of, AT.precision_of)
    assert len(calls) == n
    path = tmp_path / "tune.json"
    t.save(str(path))
    t2 = AT.Autotuner()
    t2.load(str(path))
    assert t2.table == t.table


def test_untuned_class_falls_back_to_the_default():
    t = AT.Autotuner()
    assert t.choice(fv.FV_FP64, 37, 1000) == AT.DEFAULT[fv.FV_FP64]
    assert t.choice(fv.FV_MIXED, 331, 10 ** 5) == AT.DEFAULT[fv.FV_MIXED]


def test_batch_workload_shape():
    slices = W.config_batch(seed=4, n_slices=64)
    n_ant = {len(s.problem.ant_enu) for s in slices}
    assert n_ant <= {37, 61, 91, 127, 169, 217, 271, 331}
    for s in slices:
        p = s.problem
        assert 1000 <= p.sky.n_src <= 500000
        assert p.eps in (1e-6, 1e-9)
        assert s.precision == ("mixed" if p.eps >= 1e-6 else "fp64")
        assert s.nufft_eps == (p.eps if s.precision == "mixed" else 0.1 * p.eps)
        assert len(p.freqs_hz) == 1 and len(p.lsts_rad) == 1
        assert 100e6 <= p.freqs_hz[0] <= 200e6
        assert p.sky.flux.shape == (1, p.sky.n_src, 1)
        assert len(p.pairs) == len(p.ant_enu) * (len(p.ant_enu) - 1) // 2
    # the skies are prefixes of one catalogue
    a, b = sorted(slices, key=lambda s: s.problem.sky.n_src)[:2]
    n = a.problem.sky.n_src
    assert (a.problem.sky.ra == b.problem.sky.ra[:n]).all()


def test_bin_shapes_are_tuned_for_a_type3_gather_winner():
    calls = []

    def timer(choice, bs):
        calls.append(choice)
        t = 1.0 if (choice.transform == "type3" and choice.spread == "gather" and choice.fft_max_radix == 8
                    and choice.upsampfac == 2.0) else 2.0
        if tuple(choice.bin_size) == (4, 4):
            t = 0.5
        return t, ("lattice" if choice.transform == "auto" else "type3")

    slices = [s for s in _slices() if s.precision == "mixed"][:1]
    t = AT.Autotuner(timer, routes=("auto", "type3"))
    table = t.tune(slices, AT.key_of, AT.precision_of)
    (best,) = table.values()
    assert best == AT.Choice(2.0, "gather", 8, "type3", (4, 4))
    assert len(calls) == 16 + len(AT.BIN_SHAPES)
    assert best.plan_kwargs()["bin_size"] == (4, 4)


def test_an_auto_winner_that_took_the_lattice_route_gets_no_bin_round():
    def timer(choice, bs):
        return (1.0 if choice.transform == "auto" else 2.0), ("lattice" if choice.transform == "auto" else "type3")

    slices = [s for s in _slices() if s.precision == "fp64"][:1]
    t = AT.Autotuner(timer, routes=("auto", "type3"))
    (best,) = t.tune(slices, AT.key_of, AT.precision_of).values()
    assert best.transform == "auto" and tuple(best.bin_size) == (0, 0)
    assert len(t.timings[AT.key_of(slices[0])]) == 16


def test_default_route_set_is_auto_only_and_an_auto_type3_winner_gets_bins():
    def timer(choice, bs):
        t = 1.0 if tuple(choice.bin_size) == (8, 8) else 2.0
        return t, "type3"          # a non-lattice array: auto resolves to type-3

    slices = [s for s in _slices() if s.precision == "mixed"][:1]
    t = AT.Autotuner(timer)
    (best,) = t.tune(slices, AT.key_of, AT.precision_of).values()
    assert tuple(best.bin_size) == (8, 8) and best.transform == "type3"
    assert len(t.timings[AT.key_of(slices[0])]) == 8 + len(AT.BIN_SHAPES)
