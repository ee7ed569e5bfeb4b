"""Pins of the oracle's dual arithmetic (Sec. 2, Eqs. 1-4) and the Sec. 3 test function."""
import math
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden_testfn():
    rows = [l for l in open(os.path.join(HERE, "golden", "testfn_sec3.txt")) if not l.startswith("#")]
    return np.array([float(v) for v in rows[0].split()])


def test_testfn_closed_form():
    x1, x2, x3, x4, x5 = 3.0, 0.1, 0.1, 1.0, 1.0
    q = x1 / x2
    f = x3 * (2 * math.cos(q) + q + math.exp(x2)) + 2 * x4 + math.sinh(x4) + x5 ** 2
    d = [x3 * (1 - 2 * math.sin(q)) / x2,
         x3 * (x1 * (2 * math.sin(q) - 1) / x2 ** 2 + math.exp(x2)),
         2 * math.cos(q) + q + math.exp(x2),
         2 + math.cosh(x4),
         2 * x5]
    got = oracle.testfn([x1, x2, x3, x4, x5])
    np.testing.assert_allclose(got, [f] + d, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(got, _golden_testfn(), rtol=1e-14)


def _complex_step(fn, f):
    """Directional derivatives of fn along each derivative channel of the dual f, by complex step."""
    h = 1e-30
    out = [fn(complex(f[0], 0.0)).real]
    for k in range(1, f.size):
        out.append(fn(complex(f[0], h * f[k])).imag / h)
    return np.array(out)


@pytest.mark.parametrize("op,fn,lo", [
    ("sqrt", np.sqrt, 0.1), ("sin", np.sin, -3), ("cos", np.cos, -3), ("sinh", np.sinh, -2),
    ("cosh", np.cosh, -2), ("exp", np.exp, -2)])
def test_unary_rule_eq4(op, fn, lo):
    rng = np.random.default_rng(11)
    for _ in range(20):
        f = rng.uniform(-1, 1, size=9)
        f[0] = rng.uniform(lo, 3)
        got = oracle.dual_op(op, f)
        np.testing.assert_allclose(got, _complex_step(fn, f), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
def test_binary_rules_eq1_3(op):
    rng = np.random.default_rng(12)
    fns = {"add": lambda a, b: a + b, "sub": lambda a, b: a - b, "mul": lambda a, b: a * b,
           "div": lambda a, b: a / b}
    for _ in range(20):
        f = rng.uniform(-2, 2, size=8)
        g = rng.uniform(-2, 2, size=8)
        g[0] = rng.choice([-1, 1]) * rng.uniform(0.3, 2)
        got = oracle.dual_op(op, f, g)
        h = 1e-30
        exp = [fns[op](complex(f[0]), complex(g[0])).real]
        for k in range(1, 8):
            exp.append(fns[op](complex(f[0], h * f[k]), complex(g[0], h * g[k])).imag / h)
        np.testing.assert_allclose(got, exp, rtol=1e-13, atol=1e-14)


def test_value_never_depends_on_derivatives():
    rng = np.random.default_rng(13)
    f = rng.uniform(0.5, 2, size=8)
    g = rng.uniform(0.5, 2, size=8)
    for op in ["add", "sub", "mul", "div", "sqrt", "sin", "cos", "sinh", "cosh", "exp"]:
        a = oracle.dual_op(op, f, g)
        b = oracle.dual_op(op, f[:1], g[:1])
        assert a[0] == b[0]
