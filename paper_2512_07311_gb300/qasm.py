"""Circuit ingestion from OpenQASM 2.0 text, and the writer for it.

The paper builds its states from circuits given as QASM files (Section 3.2, item 1). This module
reads a QASM 2.0 program into the library's gate list (`circuits.GATE_DTYPE` records plus the
matrices of general gates) and writes a gate list back out, so a circuit can come from a file
instead of the seeded generator.

Supported statements:
  OPENQASM 2.0;   include "...";   qreg name[n];   creg name[n];
  opaque name(params) args;        gate name(params) args { ... }   (declarations: skipped)
  barrier ...;    measure ...;     (no effect on the state: skipped)
  gate applications, to single qubits `q[i]` or whole registers (broadcast, as QASM 2.0 defines it)
Rejected with the line number: reset, if, gates on three or more qubits, names not listed
below, qubits outside their register, malformed parameters.

Gates:
  the paper's family (Section 3.1): sqrt_x, sqrt_y, sqrt_w (the library's SQRT_X/Y/W kinds) and
    fsim(theta, phi) (FSIM); a `_dg` suffix (sqrt_x_dg, fsim_dg, ...) sets the adjoint flag;
  the standard gates of qelib1.inc and common extensions, by their textbook matrices:
    id, x, y, z, h, s, sdg, t, tdg, sx, sxdg, rx, ry, rz, u1, p, u2, u3, u, U,
    cx, CX, cy, cz, ch, swap, iswap, crx, cry, crz, cu1, cp, cu3, rxx, ryy, rzz;
    each becomes a general 1-qubit (U1) or 2-qubit (U2) gate with its matrix;
  u1q(8 reals) and u2q(32 reals): a general 2x2 / 4x4 matrix, row-major (re, im) pairs, which
    the writer uses for the library's own U1/U2 gates.
A 4x4 matrix acts with local index b(first qubit) + 2 b(second qubit), the library's order.
Parameters are expressions of numbers, pi, + - * / ^ and sin, cos, tan, exp, ln, sqrt.
"""
from __future__ import annotations

import ast
import math
import operator
import re

import numpy as np

from . import circuits as C

_R2 = 1.0 / math.sqrt(2.0)


class QasmError(ValueError):
    """A statement the reader cannot take, with its line number."""

    def __init__(self, line: int, msg: str):
        super().__init__(f"line {line}: {msg}")
        self.line = line


# ---------------------------------------------------------------- parameter expressions

_FUNCS = {"sin": math.sin, "cos": math.cos, "tan": math.tan, "exp": math.exp, "ln": math.log, "sqrt": math.sqrt}
_BINOPS = {ast.Add: operator.add, ast.Sub: operator.sub, ast.Mult: operator.mul, ast.Div: operator.truediv,
           ast.Pow: operator.pow}


def eval_param(text: str) -> float:
    """Value of a QASM 2.0 parameter expression (no names but pi and the six functions)."""
    src = text.strip().replace("^", "**")
    if not src:
        raise ValueError("empty parameter")
    tree = ast.parse(src, mode="eval")

    def ev(node):
        if isinstance(node, ast.Expression):
            return ev(node.body)
        if isinstance(node, ast.Constant) and isinstance(node.value, (int, float)) and not isinstance(node.value, bool):
            return float(node.value)
        if isinstance(node, ast.Name) and node.id == "pi":
            return math.pi
        if isinstance(node, ast.UnaryOp) and isinstance(node.op, (ast.USub, ast.UAdd)):
            v = ev(node.operand)
            return -v if isinstance(node.op, ast.USub) else v
        if isinstance(node, ast.BinOp) and type(node.op) in _BINOPS:
            return _BINOPS[type(node.op)](ev(node.left), ev(node.right))
        if (isinstance(node, ast.Call) and isinstance(node.func, ast.Name) and node.func.id in _FUNCS
                and len(node.args) == 1 and not node.keywords):
            return _FUNCS[node.func.id](ev(node.args[0]))
        raise ValueError(f"not a parameter expression: {text!r}")

    v = ev(tree)
    if not math.isfinite(v):
        raise ValueError(f"parameter is not finite: {text!r}")
    return v


# ---------------------------------------------------------------- standard gate matrices

def _u3(theta, phi, lam):
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -np.exp(1j * lam) * s], [np.exp(1j * phi) * s, np.exp(1j * (phi + lam)) * c]])


def _rx(t):
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array([[c, -1j * s], [-1j * s, c]])


def _ry(t):
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array([[c, -s], [s, c]], dtype=complex)


def _rz(t):
    return np.diag([np.exp(-0.5j * t), np.exp(0.5j * t)])


_X = np.array([[0, 1], [1, 0]], dtype=complex)
_Y = np.array([[0, -1j], [1j, 0]])
_Z = np.diag([1.0 + 0j, -1.0])
_I2 = np.eye(2, dtype=complex)
_SX = 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]])

# name -> (number of parameters, matrix function of the parameters)
_ONE = {
    "id": (0, lambda: _I2), "x": (0, lambda: _X), "y": (0, lambda: _Y), "z": (0, lambda: _Z),
    "h": (0, lambda: _R2 * np.array([[1, 1], [1, -1]], dtype=complex)),
    "s": (0, lambda: np.diag([1, 1j])), "sdg": (0, lambda: np.diag([1, -1j])),
    "t": (0, lambda: np.diag([1, np.exp(0.25j * math.pi)])), "tdg": (0, lambda: np.diag([1, np.exp(-0.25j * math.pi)])),
    "sx": (0, lambda: _SX), "sxdg": (0, lambda: _SX.conj().T),
    "rx": (1, _rx), "ry": (1, _ry), "rz": (1, _rz),
    "u1": (1, lambda l: np.diag([1, np.exp(1j * l)])), "p": (1, lambda l: np.diag([1, np.exp(1j * l)])),
    "u2": (2, lambda p, l: _u3(math.pi / 2, p, l)), "u3": (3, _u3), "u": (3, _u3), "U": (3, _u3),
}


def _controlled(m2):
    """4x4 matrix of a gate controlled by the first qubit (local bit 0) on the second (bit 1)."""
    m = np.eye(4, dtype=complex)
    # local index j = b(first) + 2 b(second): the first qubit set means j in {1, 3}
    m[np.ix_([1, 3], [1, 3])] = m2
    return m


def _two_pauli(p, t):
    """exp(-i t/2 P (x) P) for the Pauli matrix P."""
    pp = np.kron(p, p)
    return math.cos(t / 2) * np.eye(4) - 1j * math.sin(t / 2) * pp


_SWAP = np.eye(4, dtype=complex)[[0, 2, 1, 3]]
_ISWAP = np.array([[1, 0, 0, 0], [0, 0, 1j, 0], [0, 1j, 0, 0], [0, 0, 0, 1]])

_TWO = {
    "cx": (0, lambda: _controlled(_X)), "CX": (0, lambda: _controlled(_X)), "cy": (0, lambda: _controlled(_Y)),
    "cz": (0, lambda: _controlled(_Z)), "ch": (0, lambda: _controlled(_ONE["h"][1]())),
    "swap": (0, lambda: _SWAP), "iswap": (0, lambda: _ISWAP),
    "crx": (1, lambda t: _controlled(_rx(t))), "cry": (1, lambda t: _controlled(_ry(t))),
    "crz": (1, lambda t: _controlled(_rz(t))),
    "cu1": (1, lambda l: _controlled(np.diag([1, np.exp(1j * l)]))),
    "cp": (1, lambda l: _controlled(np.diag([1, np.exp(1j * l)]))),
    "cu3": (3, lambda t, p, l: _controlled(_u3(t, p, l))),
    "rxx": (1, lambda t: _two_pauli(_X, t)), "ryy": (1, lambda t: _two_pauli(_Y, t)),
    "rzz": (1, lambda t: _two_pauli(_Z, t)),
}

_FAMILY = {"sqrt_x": C.SQRT_X, "sqrt_y": C.SQRT_Y, "sqrt_w": C.SQRT_W}


# ---------------------------------------------------------------- reader

_STMT_RE = re.compile(r"^([A-Za-z_][A-Za-z0-9_]*)\s*(\((.*)\))?\s*(.*)$", re.S)
_ARG_RE = re.compile(r"^([A-Za-z_][A-Za-z0-9_]*)\s*(\[\s*(\d+)\s*\])?$")


def _split_params(text: str) -> list[str]:
    out, depth, cur = [], 0, ""
    for ch in text:
        if ch == "," and depth == 0:
            out.append(cur)
            cur = ""
            continue
        depth += ch == "("
        depth -= ch == ")"
        cur += ch
    out.append(cur)
    return [p for p in (x.strip() for x in out)] if text.strip() else []


def _statements(text: str):
    """(line, statement) pairs: comments removed, statements split at ';', gate bodies kept whole."""
    clean = []
    for ln, line in enumerate(text.splitlines(), 1):
        line = line.split("//", 1)[0]
        clean.append((ln, line))
    buf, start, depth = "", None, 0
    for ln, line in clean:
        for ch in line:
            if start is None and not ch.isspace():
                start = ln
            if ch == "{":
                depth += 1
            if ch == "}":
                depth -= 1
                if depth == 0:
                    buf += ch
                    yield start, buf.strip()
                    buf, start = "", None
                    continue
            if ch == ";" and depth == 0:
                yield start, buf.strip()
                buf, start = "", None
                continue
            if start is not None:
                buf += ch
        if start is not None:
            buf += "\n"
    if buf.strip():
        raise QasmError(start, f"statement not terminated by ';': {buf.strip()[:40]!r}")


def parse_qasm(text: str):
    """Reads an OpenQASM 2.0 program. Returns (n_qubits, gates, umats): gates is a GATE_DTYPE
    array in program order, umats maps the index of every general (U1/U2) gate to its matrix.
    Qubits are numbered over the quantum registers in declaration order."""
    qregs: dict[str, tuple[int, int]] = {}  # name -> (first qubit, size)
    cregs: set[str] = set()
    n = 0
    recs, umats = [], {}
    seen_header = False

    def qubits_of(ln, arg):
        m = _ARG_RE.match(arg.strip())
        if not m:
            raise QasmError(ln, f"bad qubit argument {arg.strip()!r}")
        name, idx = m.group(1), m.group(3)
        if name not in qregs:
            raise QasmError(ln, f"unknown quantum register {name!r}")
        first, size = qregs[name]
        if idx is None:
            return [first + i for i in range(size)]
        i = int(idx)
        if i >= size:
            raise QasmError(ln, f"qubit {name}[{i}] outside the register (size {size})")
        return [first + i]

    for ln, st in _statements(text):
        if not st:
            continue
        head = st.split(None, 1)[0]
        if head == "OPENQASM":
            ver = st.split(None, 1)[1].strip() if len(st.split(None, 1)) > 1 else ""
            if not ver.startswith("2"):
                raise QasmError(ln, f"OpenQASM version {ver!r}: only 2.x is read")
            seen_header = True
            continue
        if head in ("include",):
            continue
        if head in ("qreg", "creg"):
            m = re.match(r"^(qreg|creg)\s+([A-Za-z_][A-Za-z0-9_]*)\s*\[\s*(\d+)\s*\]$", st)
            if not m:
                raise QasmError(ln, f"bad register declaration {st!r}")
            name, size = m.group(2), int(m.group(3))
            if name in qregs or name in cregs:
                raise QasmError(ln, f"register {name!r} declared twice")
            if head == "qreg":
                if size < 1:
                    raise QasmError(ln, "empty quantum register")
                qregs[name] = (n, size)
                n += size
            else:
                cregs.add(name)
            continue
        if head in ("opaque", "gate", "barrier", "measure"):
            continue
        if head in ("reset", "if"):
            raise QasmError(ln, f"{head!r} is not a unitary operation")
        m = _STMT_RE.match(st)
        if not m:
            raise QasmError(ln, f"cannot read {st[:40]!r}")
        name, ptext, argtext = m.group(1), m.group(3), m.group(4)
        try:
            params = [eval_param(p) for p in _split_params(ptext)] if ptext is not None else []
        except (ValueError, SyntaxError, ZeroDivisionError, OverflowError) as e:
            raise QasmError(ln, f"gate {name!r}: {e}") from None
        args = [a for a in argtext.split(",")] if argtext.strip() else []
        qlists = [qubits_of(ln, a) for a in args]
        flags = 0
        base = name
        if name.endswith("_dg") and name[:-3] in (*_FAMILY, "fsim"):
            base, flags = name[:-3], C.ADJOINT
        if base in _FAMILY or base == "fsim" or name in _ONE or name in _TWO or name in ("u1q", "u2q"):
            nq = 2 if (base == "fsim" or name in _TWO or name == "u2q") else 1
        else:
            raise QasmError(ln, f"unknown gate {name!r}")
        if len(qlists) != nq:
            raise QasmError(ln, f"gate {name!r} takes {nq} qubit argument(s), got {len(qlists)}")
        # broadcast: registers of one size, single qubits repeated
        width = max(len(x) for x in qlists)
        if any(len(x) not in (1, width) for x in qlists):
            raise QasmError(ln, f"gate {name!r}: registers of different sizes")
        for r in range(width):
            qs = [x[0] if len(x) == 1 else x[r] for x in qlists]
            if nq == 2 and qs[0] == qs[1]:
                raise QasmError(ln, f"gate {name!r} on one qubit twice")
            if base in _FAMILY:
                if params:
                    raise QasmError(ln, f"gate {name!r} takes no parameters")
                recs.append((_FAMILY[base], 1, flags, qs[0], -1, 0.0, 0.0, 0))
            elif base == "fsim":
                if len(params) != 2:
                    raise QasmError(ln, "fsim takes two parameters (theta, phi)")
                recs.append((C.FSIM, 2, flags, qs[0], qs[1], params[0], params[1], 0))
            elif name in ("u1q", "u2q"):
                d = 2 if name == "u1q" else 4
                if len(params) != 2 * d * d:
                    raise QasmError(ln, f"{name} takes {2 * d * d} parameters")
                mat = (np.array(params[0::2]) + 1j * np.array(params[1::2])).reshape(d, d)
                umats[len(recs)] = mat
                recs.append((C.U1 if d == 2 else C.U2, nq, 0, qs[0], qs[1] if nq == 2 else -1, 0.0, 0.0, 0))
            else:
                table = _ONE if nq == 1 else _TWO
                npar, fn = table[name]
                if len(params) != npar:
                    raise QasmError(ln, f"gate {name!r} takes {npar} parameter(s), got {len(params)}")
                mat = np.asarray(fn(*params), dtype=np.complex128)
                umats[len(recs)] = mat
                recs.append((C.U1 if nq == 1 else C.U2, nq, 0, qs[0], qs[1] if nq == 2 else -1, 0.0, 0.0, 0))
    if not seen_header:
        raise QasmError(1, "missing 'OPENQASM 2.0;' header")
    if n == 0:
        raise QasmError(1, "no quantum register")
    return n, C.gate_array(recs), umats


def read_qasm(path: str):
    with open(path) as f:
        return parse_qasm(f.read())


# ---------------------------------------------------------------- writer

_KIND_NAME = {C.SQRT_X: "sqrt_x", C.SQRT_Y: "sqrt_y", C.SQRT_W: "sqrt_w"}


def to_qasm(n_qubits: int, gates: np.ndarray, umats: dict | None = None, reg: str = "q") -> str:
    """OpenQASM 2.0 text of a gate list (the library's kinds, with their angles written
    exactly). General gates (U1/U2) become u1q/u2q with their matrices."""
    umats = umats or {}
    lines = ["OPENQASM 2.0;", 'include "qelib1.inc";',
             "opaque sqrt_x a;", "opaque sqrt_y a;", "opaque sqrt_w a;", "opaque fsim(theta, phi) a, b;",
             "opaque sqrt_x_dg a;", "opaque sqrt_y_dg a;", "opaque sqrt_w_dg a;", "opaque fsim_dg(theta, phi) a, b;",
             f"qreg {reg}[{n_qubits}];"]
    declared_u = set()
    for i, g in enumerate(np.asarray(gates, dtype=C.GATE_DTYPE)):
        kind, flags, q0, q1 = int(g["kind"]), int(g["flags"]), int(g["q0"]), int(g["q1"])
        dg = "_dg" if flags & C.ADJOINT else ""
        if kind in _KIND_NAME:
            lines.append(f"{_KIND_NAME[kind]}{dg} {reg}[{q0}];")
        elif kind == C.FSIM:
            lines.append(f"fsim{dg}({float(g['theta'])!r}, {float(g['phi'])!r}) {reg}[{q0}], {reg}[{q1}];")
        elif kind in (C.U1, C.U2):
            if i not in umats:
                raise ValueError(f"gate {i}: general gate without a matrix")
            mat = np.asarray(umats[i], dtype=np.complex128)
            if flags & C.ADJOINT:
                mat = mat.conj().T
            name = "u1q" if kind == C.U1 else "u2q"
            if name not in declared_u:
                npar = 8 if kind == C.U1 else 32
                lines.insert(10 + len(declared_u), f"opaque {name}({', '.join(f'p{k}' for k in range(npar))}) "
                             + ("a;" if kind == C.U1 else "a, b;"))
                declared_u.add(name)
            vals = ", ".join(f"{float(x)!r}" for z in mat.reshape(-1) for x in (z.real, z.imag))
            qs = f"{reg}[{q0}]" if kind == C.U1 else f"{reg}[{q0}], {reg}[{q1}]"
            lines.append(f"{name}({vals}) {qs};")
        else:
            raise ValueError(f"gate {i}: unknown kind {kind}")
    return "\n".join(lines) + "\n"


def write_qasm(path: str, n_qubits: int, gates: np.ndarray, umats: dict | None = None) -> None:
    with open(path, "w") as f:
        f.write(to_qasm(n_qubits, gates, umats))
