"""Oracle for the general elementwise front end (test infrastructure only).

The paper's input is a loop domain plus instructions (Section 2.1); the meaning of
one assignment over a rectangular domain { [i0, i1, ...] : 0 <= ik < nk } is that it
is executed once for every point of the domain (Section 2.3: in no particular order,
since no point reads what another writes).  This module evaluates such an assignment
directly from its text: Python's own parser reads the statement (the instruction
syntax ``z[i] = a*x[i] + y[i]`` is also a Python statement), and each operation is
applied to whole float32 arrays with numpy, so every +, -, * and / is one IEEE
single-precision operation rounded to nearest-even, in the order the expression
tree gives.  Array accesses index by a subset of the domain's inames in domain order
(``c[j]`` inside a domain over [i, j] is broadcast along i); names that are not
indexed are scalar parameters.

It shares no code with the library (the library parses with its own C++ code and
compiles the instruction to a CUDA kernel).
"""

from __future__ import annotations

import ast

import numpy as np

_OPS = {ast.Add: np.add, ast.Sub: np.subtract, ast.Mult: np.multiply, ast.Div: np.divide}


def _index_names(sub: ast.Subscript):
    sl = sub.slice
    elts = sl.elts if isinstance(sl, ast.Tuple) else [sl]
    names = []
    for e in elts:
        if not isinstance(e, ast.Name):
            raise ValueError("array indices must be inames")
        names.append(e.id)
    return names


def evaluate(instruction: str, inames, sizes, arrays: dict, scalars: dict | None = None,
             dtype=np.float32) -> np.ndarray:
    """Evaluate ``lhs[inames] = expr`` over the domain with extents ``sizes``.

    arrays: name -> numpy array whose shape is the extents of the inames it is indexed by.
    scalars: name -> number. Returns the output array (shape ``sizes``) in ``dtype``.
    """
    scalars = scalars or {}
    inames = list(inames)
    sizes = [int(n) for n in sizes]
    tree = ast.parse(instruction.strip(), mode="exec")
    if len(tree.body) != 1 or not isinstance(tree.body[0], ast.Assign) or len(tree.body[0].targets) != 1:
        raise ValueError("expected one assignment")
    target, value = tree.body[0].targets[0], tree.body[0].value
    if not isinstance(target, ast.Subscript) or _index_names(target) != inames:
        raise ValueError("the output must be indexed by every iname, in domain order")

    def access(sub: ast.Subscript):
        names = _index_names(sub)
        pos = [inames.index(n) for n in names]
        if pos != sorted(pos) or len(set(pos)) != len(pos):
            raise ValueError("indices must follow the domain order")
        a = np.asarray(arrays[sub.value.id], dtype=dtype)
        if a.shape != tuple(sizes[p] for p in pos):
            raise ValueError(f"array {sub.value.id} has shape {a.shape}")
        shape = [sizes[k] if k in pos else 1 for k in range(len(inames))]
        return a.reshape(shape)

    def ev(node):
        if isinstance(node, ast.BinOp) and type(node.op) in _OPS:
            return _OPS[type(node.op)](ev(node.left), ev(node.right), dtype=dtype)
        if isinstance(node, ast.UnaryOp) and isinstance(node.op, ast.USub):
            return np.negative(ev(node.operand), dtype=dtype)
        if isinstance(node, ast.UnaryOp) and isinstance(node.op, ast.UAdd):
            return ev(node.operand)
        if isinstance(node, ast.Constant) and isinstance(node.value, (int, float)):
            return dtype(node.value)
        if isinstance(node, ast.Name):
            return dtype(scalars[node.id])
        if isinstance(node, ast.Subscript):
            return access(node)
        raise ValueError(f"unsupported expression: {ast.dump(node)}")

    with np.errstate(all="ignore"):
        out = ev(value)
    return np.ascontiguousarray(np.broadcast_to(np.asarray(out, dtype=dtype), tuple(sizes)))
