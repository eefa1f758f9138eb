"""The seeded synthetic workloads have the shapes their names and descriptions state."""

import numpy as np

from workload import gen, make_workload, mutate, random_sequences


def test_generator_is_deterministic():
    a = random_sequences(11, 300, 300, 0.5, 20, 1000)
    b = random_sequences(11, 300, 300, 0.5, 20, 1000)
    assert (a.residues == b.residues).all() and (a.offsets == b.offsets).all()
    assert a.residues.max() < 20
    L = a.lengths
    assert L.min() >= 20 and L.max() <= 1000


def test_workload_shapes_small():
    w1 = make_workload("one_query_vs_2k")
    assert len(w1["db"]) == 2000 and w1["queries"].lengths.tolist() == [144]
    cells = w1["db"].total * 144
    assert 0.8e8 < cells < 1.2e8  # "~1e8 cells"
    assert gen.twenty_query_lengths()[0] == 144 and gen.twenty_query_lengths()[-1] == 5478
    w3 = make_workload("homologs_8k")
    assert len(w3["db"]) == 2010 and w3["queries"].lengths.tolist() == [144, 8000]
    assert len(w3["homolog_ids"]) == 10
    for i in w3["homolog_ids"]:
        assert 7500 < len(w3["db"][int(i)]) < 8500
    w4 = make_workload("thousand_queries_vs_50k", n_db=1000, n_queries=50)
    assert len(w4["queries"]) == 50
    assert w4["queries"].lengths.min() >= 50 and w4["queries"].lengths.max() <= 2000
    w5 = make_workload("serving_500k", n_db=1000, n_queries=100)
    arr = w5["arrivals"]
    assert (np.diff(arr) > 0).all() and 0.5 < arr[-1] / 100 * 50 < 2.0


def test_mutation_model_identity():
    rng = np.random.Generator(np.random.PCG64(1))
    src = rng.integers(0, 20, size=4000).astype(np.uint8)
    hom = mutate(np.random.Generator(np.random.PCG64(2)), src)
    assert abs(len(hom) - len(src)) < 200
    # roughly 90% identity along the unshifted prefix before the first indel
    same = (hom[:30] == src[:30]).mean()
    assert same > 0.6


def test_query_batch_144():
    from workload import query_batch_144

    a, b = query_batch_144(8), query_batch_144(8)
    assert np.array_equal(a.residues, b.residues) and a.lengths.tolist() == [144] * 8
    assert a.residues.max() < 20 and len({bytes(a[i]) for i in range(8)}) == 8
