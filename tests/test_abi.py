"""The C-ABI library loads and exports every function include/plastic_arbor.h
declares; the binding's struct layouts match the header.  No GPU needed."""
import ctypes as C
import os
import re

from paper_2411_16445_b300 import build_lib
from paper_2411_16445_b300 import engine as E

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "plastic_arbor.h")) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"\b(pa_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    build_lib.build()
    lib = E.lib()
    names = declared_functions()
    assert "pa_build_model" in names and "pa_advance" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in the header but not exported"
    assert set(E.EXPORTED) <= set(names)


def test_struct_layouts_match_header():
    assert E.CELL_DTYPE.itemsize == 72
    assert E.CONN_DTYPE.itemsize == 48
    assert C.sizeof(E.Morph) == 40
    assert C.sizeof(E.Mech) == 16
    assert C.sizeof(E.Options) == 80
    assert C.sizeof(E.Info) == 88
    assert C.sizeof(E.KernelStats) == 40


def test_last_error_without_gpu_is_a_string():
    msg = E.lib().pa_last_error()
    assert isinstance(msg, bytes)


def test_build_rejects_bad_arguments_before_touching_the_device():
    """Descriptor validation happens on the host, so it is testable without a GPU."""
    from paper_2411_16445_b300 import workloads as W
    import pytest
    net = W.single_neuron()
    net.conn_mech = net.conn_mech.copy()
    net.conn_mech[0] = 0  # the HH density mechanism is not a synapse
    with pytest.raises(E.PaError) as ei:
        E.Model(net)
    assert ei.value.code == -1 and "synapse" in str(ei.value)
