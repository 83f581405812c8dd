"""The Python binding's argument marshalling, on CPU: shapes, row counts,
dimensions and variant names are checked before any call into the library,
and a bad one raises (no GPU is needed for that)."""
import numpy as np
import pytest

import paper_1907_04839_gb300 as gsh


def z(n, d=3):
    return np.zeros((n, d), np.float32)


@pytest.mark.parametrize("q0,p0,target,msg", [
    (z(10), z(10), z(9), "target: expected 10 rows"),
    (z(10), z(9), z(10), "p0: expected 10 rows"),
    (z(10, 4), z(10, 4), z(10, 4), "expected shape (N, 3)"),
    (z(10), z(10, 2), z(10), "expected shape (N, 3)"),
    (z(10, 2), z(10), z(10, 2), "expected shape (N, 2)"),
    (np.zeros(30, np.float32), z(10), z(10), "expected shape (N, 3)"),
])
def test_shoot_gradient_rejects_mismatched_arrays(q0, p0, target, msg):
    with pytest.raises(ValueError, match=msg.replace("(", r"\(").replace(")", r"\)")):
        gsh.shoot_gradient(q0, p0, target, 4, 0.1, 10.0)


def test_shoot_forward_rejects_mismatched_arrays():
    with pytest.raises(ValueError, match="p0: expected 5 rows"):
        gsh.shoot_forward(z(5), z(6), 4, 0.1)


@pytest.mark.parametrize("kw,msg", [({"integrator": "rk5"}, "integrator must be one of"),
                                    ({"h_at": "middle"}, "h_at must be one of")])
def test_unknown_variant_names_are_rejected(kw, msg):
    with pytest.raises(ValueError, match=msg):
        gsh.shoot_gradient(z(4), z(4), z(4), 4, 0.1, 10.0, **kw)
    if "integrator" in kw:
        with pytest.raises(ValueError, match=msg):
            gsh.shoot_forward(z(4), z(4), 4, 0.1, **kw)


def test_register_rejects_a_wrong_initial_momentum():
    with pytest.raises(ValueError, match="p0: expected shape"):
        gsh.register(z(8), z(8), 4, 0.1, 10.0, p0=z(7))
