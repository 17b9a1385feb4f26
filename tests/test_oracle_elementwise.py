"""Pins for the elementwise-instruction oracle (oracle/elementwise.py): hand-worked cases,
closed forms of saxpy (Table 1's streaming workload), single-precision rounding of every
operation checked against torch's CPU float32 arithmetic (an independent library), numpy's
outer operations for broadcasting, and planted mistakes that the pins must catch."""

import ast
import json
import os

import numpy as np
import pytest

from oracle import elementwise as ew

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _pin_failures(fn):
    fails = []
    with open(os.path.join(GOLDEN, "elementwise_hand.json")) as fh:
        cases = json.load(fh)["cases"]
    for c in cases:
        arrays = {k: np.array(v, np.float32) for k, v in c["arrays"].items()}
        got = fn(c["instruction"], c["inames"], c["sizes"], arrays, c["scalars"])
        if not np.array_equal(got, np.array(c["out"], np.float32)):
            fails.append("hand:" + c["instruction"])
    rng = np.random.default_rng(41)
    n = 10000
    x = rng.standard_normal(n).astype(np.float32)
    y = rng.standard_normal(n).astype(np.float32)
    saxpy = "z[i] = a*x[i] + y[i]"
    if not np.array_equal(fn(saxpy, ["i"], [n], {"x": x, "y": y}, {"a": 0.0}), y):
        fails.append("a_zero")
    if not np.array_equal(fn(saxpy, ["i"], [n], {"x": x, "y": np.zeros(n, np.float32)}, {"a": 1.0}), x):
        fails.append("y_zero")
    torch = pytest.importorskip("torch")
    a = np.float32(0.7071)
    tx, ty = torch.from_numpy(x), torch.from_numpy(y)
    want = torch.add(torch.mul(tx, float(a)), ty).numpy()
    if not np.array_equal(fn(saxpy, ["i"], [n], {"x": x, "y": y}, {"a": float(a)}), want):
        fails.append("torch_saxpy")
    want = torch.div(torch.sub(tx, ty), 3.0).numpy()
    if not np.array_equal(fn("q[i] = (x[i] - y[i]) / 3", ["i"], [n], {"x": x, "y": y}, {}), want):
        fails.append("torch_div")
    c, d = rng.standard_normal(37).astype(np.float32), rng.standard_normal(11).astype(np.float32)
    if not np.array_equal(fn("b[i,j] = c[j] * d[i]", ["i", "j"], [11, 37], {"c": c, "d": d}, {}),
                          np.multiply.outer(d, c)):
        fails.append("outer")
    return fails


def test_oracle_passes_every_pin():
    assert _pin_failures(ew.evaluate) == []


def _mutant(kind):
    def fn(instruction, inames, sizes, arrays, scalars):
        if kind == "float64_then_round":
            return ew.evaluate(instruction, inames, sizes, arrays, scalars, dtype=np.float64).astype(np.float32)
        if kind == "swap_sub":
            tree = ast.parse(instruction)

            class Swap(ast.NodeTransformer):
                def visit_BinOp(self, node):
                    self.generic_visit(node)
                    if isinstance(node.op, ast.Sub):
                        node.left, node.right = node.right, node.left
                    return node
            return ew.evaluate(ast.unparse(Swap().visit(tree)), inames, sizes, arrays, scalars)
        if kind == "broadcast_wrong_axis" and len(inames) == 2:
            # a 1-D array broadcast along the other iname: read c[j] as if it were c[i]
            text = instruction.split("=", 1)
            rhs = text[1].replace("[j]", "[@]").replace("[i]", "[j]").replace("[@]", "[i]")
            return ew.evaluate(text[0] + "=" + rhs, inames, sizes, arrays, scalars)
        return ew.evaluate(instruction, inames, sizes, arrays, scalars)
    return fn


@pytest.mark.parametrize("kind", ["float64_then_round", "swap_sub", "broadcast_wrong_axis"])
def test_pins_catch_planted_mistakes(kind):
    try:
        fails = _pin_failures(_mutant(kind))
    except ValueError:
        fails = ["raised"]  # a mistake that makes the evaluation impossible is caught too
    assert fails, kind


def test_rejects_malformed_instructions():
    with pytest.raises(ValueError):
        ew.evaluate("z[j] = x[j]", ["i"], [3], {"x": np.zeros(3, np.float32)})
    with pytest.raises(ValueError):
        ew.evaluate("b[i,j] = c[j,i]", ["i", "j"], [2, 2], {"c": np.zeros((2, 2), np.float32)})
