"""Mixed-size plans on the host: validation and workspace sizing (no GPU needed)."""
import ctypes

import numpy as np
import pytest

import paper_1304_7054_gb300 as kg
from paper_1304_7054_gb300 import build as libbuild
from paper_1304_7054_gb300 import inputs


@pytest.fixture(scope="module", autouse=True)
def lib():
    libbuild.build()
    return kg.load_library()


def classes_of(v):
    return [(k, n, *cs) for (k, n), cs in zip(v.classes, v.comps)]


def test_plan_and_workspace_size():
    v = inputs.make_varlen(500, seed=1)
    p = kg.VarlenPlan(classes_of(v), v.class_of, v.x_off, v.y_off)
    ws = p.workspace_size()
    assert ws >= 500 * 16 and ws % 256 == 0
    p.close()


def test_empty_plan():
    p = kg.VarlenPlan([(2, 4, np.eye(4), np.eye(4))], [], [], [])
    assert p.workspace_size() == 0
    p.close()


@pytest.mark.parametrize("bad", ["duplicate", "class_range", "neg_offset", "overlap_y", "kind", "n0", "f64"])
def test_plan_validation(bad):
    I = np.eye(4)
    classes = [(2, 4, I, I), (3, 4, I, I, I)]
    cls, xo, yo = [0, 1, 0], [0, 16, 80], [0, 16, 80]
    io = "f32"
    if bad == "duplicate":
        classes.append((2, 4, I, I))
    if bad == "class_range":
        cls = [0, 2, 0]
    if bad == "neg_offset":
        xo = [0, -1, 80]
    if bad == "overlap_y":
        yo = [0, 8, 80]
    if bad == "kind":
        classes[1] = (4, 4, I, I, I)
    if bad == "n0":
        classes[0] = (2, 0, I, I)
    if bad == "f64":
        io = "f64"
    with pytest.raises(kg.KronError) as e:
        kg.VarlenPlan(classes, cls, xo, yo, io=io)
    assert e.value.status in (1, 2)


def test_execute_argument_checks():
    I = np.eye(4)
    p = kg.VarlenPlan([(2, 4, I, I)], [0, 0], [0, 16], [0, 16])
    L = kg.load_library()
    # workspace too small / misaligned, aliasing: rejected before any launch
    assert L.kron_varlen_execute(p.handle, 0x100000, 0x200000, 0x300000, 1, None) == 4
    assert L.kron_varlen_execute(p.handle, 0x100000, 0x200000, 0x300010, 1 << 20, None) == 4
    assert L.kron_varlen_execute(p.handle, 0x100000, 0x100000 + 64, 0x300000, 1 << 20, None) == 3
    assert L.kron_varlen_execute(p.handle, None, 0x200000, 0x300000, 1 << 20, None) == 1
    assert L.kron_varlen_execute(None, 0x100000, 0x200000, 0x300000, 1 << 20, None) == 1
    p.close()
