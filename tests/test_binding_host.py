"""The Python binding's argument checks, on the host (no GPU). The C ABI takes plain pointers
and reads as many entries as its other arguments imply, so the binding refuses, before the
call, any array or tensor shorter than that, and any tensor in the wrong memory space or type.
"""
import types

import numpy as np
import pytest

import inputs
from paper_2103_14294_b300 import huge

_NO_GRAPH = types.SimpleNamespace(handle=None)  # the checks run before the graph is used


def _einval(fn, *a, **kw):
    with pytest.raises(huge.HugeError) as ei:
        fn(*a, **kw)
    assert ei.value.code == huge.EINVAL
    return str(ei.value)


def test_query_arrays_hold_k_entries():
    k, e = inputs.QUERIES["c4"]
    assert "order" in _einval(huge.Plan, _NO_GRAPH, k, e, order=[0, 1, 3])
    assert "labels" in _einval(huge.Plan, _NO_GRAPH, k, e, order=[0, 1, 3, 2], labels=[0, 1])
    assert "order" in _einval(huge.plan_offline, k, e, order=[0, 1])
    assert "labels" in _einval(huge.plan_offline, k, e, order=[0, 1, 3, 2], labels=[0], lstart=[0, 4])
    assert "lstart" in _einval(huge.plan_offline, k, e, order=[0, 1, 3, 2], labels=[0, 0, 0, 0])
    assert "order" in _einval(huge.count_noalloc, 0, 0, 10, 20, k, e, order=[0])
    with pytest.raises(ValueError):  # one cardinality per vertex mask
        huge.plan_offline(k, e, card=np.ones(8))


def test_mlp_arrays_and_tensors_are_checked():
    torch = pytest.importorskip("torch")
    m = object.__new__(huge.MLP)  # no device state: every check runs before the call
    m.handle, m.n_params = None, huge.load().huge_mlp_num_params()
    assert "params" in _einval(m.set_params, np.zeros(10, np.float32))
    assert "mu" in _einval(m.set_params, None, np.zeros(63, np.float32), np.ones(64, np.float32))
    x = torch.zeros(4, 64)
    y = torch.zeros(4)
    assert "current CUDA device" in _einval(m.forward, x, y)  # host tensors
    assert "float32" in _einval(m.forward, x.double(), y)
    assert "shape" in _einval(m.train, torch.zeros(4, 32), y, epochs=1)
    # the tensor check itself: length before memory space, so it shows without a GPU
    assert "holds 3 entries" in _einval(huge._need_device, torch.zeros(3), 4, "y")
    assert "contiguous" in _einval(huge._need_device, torch.zeros(4, 64).t(), 0, "x")


def test_list_sink_is_a_device_tensor_of_k_columns():
    torch = pytest.importorskip("torch")
    plan = types.SimpleNamespace(k=4, handle=None)
    assert "shape" in _einval(huge.enumerate, plan, mode=huge.LIST, sink=torch.zeros((8, 3), dtype=torch.int32))
    assert "int32" in _einval(huge.enumerate, plan, mode=huge.LIST, sink=torch.zeros((8, 4)))
    assert "current CUDA device" in _einval(huge.enumerate, plan, mode=huge.LIST,
                                            sink=torch.zeros((8, 4), dtype=torch.int32))
