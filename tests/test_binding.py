"""Host-side helpers of the Python binding (no GPU): the morphology descriptor
table points at the right data, and the connection descriptors packed in
chunks on threads are byte-identical to a field-by-field fill."""
import ctypes as C

import numpy as np
import pytest

from paper_2411_16445_b300 import engine as E
from paper_2411_16445_b300 import workloads as W


def test_morph_table_layout_and_pointers():
    assert E.MORPH_DTYPE.itemsize == C.sizeof(E.Morph)
    for name, _ in E.Morph._fields_:
        assert E.MORPH_DTYPE.fields[name][1] == getattr(E.Morph, name).offset
    rng = np.random.default_rng(7)
    morphs = [W.random_binary_tree(rng, int(rng.integers(1, 30))) for _ in range(50)]
    morphs.append(W.soma_only(12.0))
    keep = []
    tab = E._morph_table(morphs, keep)
    for i, m in enumerate(morphs):
        n = int(tab["n_cv"][i])
        assert n == m.n_cv
        for f, src, ct in (("parent", "parent", C.c_int32), ("length_um", "length", C.c_double),
                           ("diam_um", "diam", C.c_double), ("region", "region", C.c_int32)):
            got = np.ctypeslib.as_array((ct * n).from_address(int(tab[f][i])))
            assert np.array_equal(got, getattr(m, src))


def test_morph_table_rejects_mismatched_lengths():
    m = W.soma_only(10.0)
    bad = W.Morphology(parent=np.array([-1, 0], np.int32), length=np.ones(3),
                       diam=np.ones(2), region=np.zeros(2, np.int32))
    with pytest.raises(ValueError):
        E._morph_table([m, bad], [])
    assert len(E._morph_table([], [])) == 1


@pytest.mark.parametrize("n", [0, 1000, 2 * (1 << 20) + 12345])
def test_pack_equals_field_fill(n):
    rng = np.random.default_rng(n)
    cols = {"src_gid": rng.integers(-1, 1000, n).astype(np.int32),
            "dst_gid": rng.integers(0, 1000, n).astype(np.int32),
            "dst_cv": rng.integers(0, 50, n).astype(np.int32),
            "mech": rng.integers(0, 4, n).astype(np.int32),
            "weight": rng.standard_normal(n), "delay_ms": rng.uniform(0.1, 5.0, n),
            "rate_hz": rng.uniform(0.0, 10.0, n),
            "poisson_id": rng.integers(-1, 1 << 40, n)}
    ref = np.zeros(n, E.CONN_DTYPE)
    for f, c in cols.items():
        ref[f] = c
    got = E._pack(E.CONN_DTYPE, n, cols)
    assert got.dtype == E.CONN_DTYPE and got.tobytes() == ref.tobytes()
