"""Planted mistakes in the oracle must fail its pins.

The oracle can only judge the GPU path if its pins catch the mistakes one
could plausibly make in it.  Each case below copies lexoracle.c, plants one
such mistake (a dropped condition of Definition 2 or 3, an off-by-one, a
first match in place of the longest, a wrong filter), compiles the copy with
gcc into a temporary directory, swaps it in for the oracle's library and runs
the oracle's fast pins: the worked examples of the paper
(test_oracle_pins.py), the hand-written pi_I streams and plans
(test_oracle_discard_plan.py) and the Python re.fullmatch cross-check
(test_oracle_re.py).  At least one pin must fail.  The planner and the
chunked run, which are Python, are replaced by mutated copies in the same
way.  The Python parts of the oracle (entry contexts, live sets, split
windows, the FP64 model) are mutated in their source text and loaded in place
of the real module before their own pins are loaded.  A control run with an
unmutated copy passes every pin, so the failures come from the planted
mistakes and not from the harness.  Pins that compare the oracle with the
product's host code (those that take the library fixture) are left out: a
mistake must be caught by what fixes the oracle, not by the product.
Nothing here runs on a GPU.
"""

import ctypes
import importlib.util
import inspect
import os
import subprocess
import sys
import types
from typing import List

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)     # some pin modules import helpers from others
PIN_MODULES = ("test_oracle_pins.py", "test_oracle_discard_plan.py", "test_oracle_re.py")


def _load_module(fname):
    spec = importlib.util.spec_from_file_location("mut_pins_" + fname[:-3], os.path.join(HERE, fname))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


PINS = [_load_module(f) for f in PIN_MODULES]


def _pin_calls(mods):
    """Every pin test of `mods` with its arguments (parametrize marks
    expanded); tests that take fixtures are skipped."""
    for mod in mods:
        for name in sorted(dir(mod)):
            if not name.startswith("test_"):
                continue
            f = getattr(mod, name)
            marks = [m for m in getattr(f, "pytestmark", []) if m.name == "parametrize"]
            params = list(inspect.signature(f).parameters)
            if not marks:
                if not params:
                    yield f"{mod.__name__}.{name}", f, ()
                continue
            assert len(marks) == 1, name
            argnames, argvalues = marks[0].args[0], marks[0].args[1]
            names = [a.strip() for a in argnames.split(",")] if isinstance(argnames, str) else list(argnames)
            if params != names:
                continue
            for v in argvalues:
                vals = getattr(v, "values", v)
                yield f"{mod.__name__}.{name}{vals}", f, tuple(vals) if len(names) > 1 else (vals,)


def _failing_pins(mods=None, first=False) -> List[str]:
    failed = []
    for name, f, args in _pin_calls(PINS if mods is None else mods):
        try:
            f(*args)
        except Exception:        # an assertion, or a mistake that breaks the caller
            failed.append(name)
            if first:
                break
    return failed


def _build_variant(tmp_path, old, new):
    src = open(oracle._SRC).read()
    if old is not None:
        assert src.count(old) == 1, f"mutation site not unique: {old!r}"
        src = src.replace(old, new)
    c = tmp_path / "lexoracle_variant.c"
    c.write_text(src)
    so = tmp_path / "liblexoracle_variant.so"
    subprocess.check_call(["gcc", *oracle.CFLAGS, "-shared", "-fPIC", str(c), oracle._SRC_PAR, "-o", str(so)])
    return oracle._bind(ctypes.CDLL(str(so)))


@pytest.fixture
def swap_library(monkeypatch):
    oracle._load()                       # the real library first, so that restoring it is exact

    def swap(lib):
        monkeypatch.setattr(oracle, "_lib", lib)
    return swap


# (name, text in lexoracle.c, replacement)
C_MUTATIONS = [
    # Section 3, the scanner
    ("first match instead of the longest",
     "last_kind = tau[q];\n            }", "last_kind = tau[q];\n                break;\n            }"),
    ("kind of the first accepting prefix kept",
     "last_kind = tau[q];", "if (last_kind == UNDEF) last_kind = tau[q];"),
    ("token length off by one", "lens[count] = last - i;", "lens[count] = last - i + 1;"),
    ("lexing error skipped instead of halting",
     "if (last < 0)\n            break;", "if (last < 0) {\n            i++;\n            continue;\n        }"),
    # Section 5, pi_I
    ("discarded kinds kept", "in_I[t])\n            continue;", "in_I[t] && 0)\n            continue;"),
    ("kept and discarded kinds swapped", "in_I[t])\n            continue;", "!in_I[t])\n            continue;"),
    # Section 4, Q+
    ("Q+ without co-accessibility", "live[q] = reach[q] && coacc[q];", "live[q] = reach[q];"),
    ("Q+ without reachability", "live[q] = reach[q] && coacc[q];", "live[q] = coacc[q];"),
    ("co-accessibility seeded empty", "coacc[q] = tau[q] != UNDEF;", "coacc[q] = 0;"),
    # Definition 1
    ("re-entrancy through the empty word", "reentrant = back[q0];", "reentrant = 1;"),
    ("re-entrancy never detected", "reentrant = back[q0];", "reentrant = 0;"),
    # Definition 2
    ("exact condition allows states other than q0", "if (q != q0)\n                ex = 0;", ""),
    ("exact condition ignores re-entrancy", "if (d0 != UNDEF && reentrant)\n            ex = 0;", ""),
    # Definition 3
    ("A(q) ignores re-entrancy", "int A = (q == q0) && !reentrant;", "int A = (q == q0);"),
    ("C(q) without tau(q) defined", "(tau[q] != UNDEF) && (d0 != UNDEF)", "(d0 != UNDEF)"),
    ("C(q) without delta+(q0, b) = delta+(q, b)", "(d0 != UNDEF) && (d0 == t) && only_I[q]",
     "(d0 != UNDEF) && only_I[q]"),
    ("C(q) without T(q) inside I", "(d0 == t) && only_I[q];", "(d0 == t);"),
    ("T(q) counts non-accepting states", "if (!seen[p] || tau[p] == UNDEF)\n                continue;",
     "if (!seen[p])\n                continue;"),
    # Corollary 2 / Proposition 2
    ("exact useful set without delta+(q0, b) defined",
     "exact_use[b] = (uint8_t)(ex && d0 != UNDEF);", "exact_use[b] = (uint8_t)ex;"),
    ("modulo useful set without delta+(q0, b) defined",
     "modulo_use[b] = (uint8_t)(mo && d0 != UNDEF);", "modulo_use[b] = (uint8_t)mo;"),
]


def test_unmutated_copy_passes_every_pin(tmp_path, swap_library):
    swap_library(_build_variant(tmp_path, None, None))
    assert _failing_pins() == []


@pytest.mark.parametrize("name,old,new", C_MUTATIONS, ids=[m[0] for m in C_MUTATIONS])
def test_planted_mistake_in_the_c_oracle_fails_a_pin(tmp_path, swap_library, name, old, new):
    swap_library(_build_variant(tmp_path, old, new))
    assert _failing_pins(), f"no pin catches: {name}"


# Section 6, the planner: mutated copies of oracle.plan

def _plan_variant(kind):
    def plan(data, useful, k):
        w = oracle._as_bytes(data)
        n = int(w.size)
        if k <= 1 or n == 0 or not np.any(useful):
            return []
        is_cert = np.asarray(useful, dtype=bool)[w]
        cuts = []
        for i in range(1, k):
            t = (n * i) // (k + 1) if kind == "targets" else (n * i) // k
            if kind == "backward":
                while t > 0 and not is_cert[t]:
                    t -= 1
            else:
                while t < n and not is_cert[t]:
                    t += 1
                if kind == "past the byte" and t < n:
                    t += 1
            if kind == "duplicates kept":
                if 0 < t < n:
                    cuts.append(t)
            elif 0 < t < n and (not cuts or cuts[-1] < t):
                cuts.append(t)
        return cuts
    return plan


@pytest.mark.parametrize("kind", ["backward", "targets", "past the byte", "duplicates kept"])
def test_planted_mistake_in_the_planner_fails_a_pin(monkeypatch, kind):
    monkeypatch.setattr(oracle, "plan", _plan_variant(kind))
    assert _failing_pins(), f"no pin catches the planner mistake: {kind}"


def test_chunked_run_that_ignores_a_failing_chunk_fails_a_pin(monkeypatch):
    def lex_chunks(dfa, data, cuts):
        a = oracle._as_automaton(dfa)
        w = oracle._as_bytes(data)
        bounds = [0] + sorted(int(c) for c in cuts) + [int(w.size)]
        ks, ls = [], []
        for lo, hi in zip(bounds[:-1], bounds[1:]):
            k, l, _ = oracle.lex(a, w[lo:hi])
            ks.append(k)
            ls.append(l)
        return np.concatenate(ks), np.concatenate(ls), int(w.size)
    monkeypatch.setattr(oracle, "lex_chunks", lex_chunks)
    assert _failing_pins(), "no pin catches a chunked run that reads past a failing chunk"


# The Python submodules of the oracle: mutated source text, loaded in place
# of the real module, then that module's own pins loaded against it.

SUB_PINS = {"contexts": "test_oracle_contexts.py", "live": "test_oracle_live.py",
            "windows": "test_oracle_windows.py", "model": "test_oracle_model.py"}


def _swap_submodule(monkeypatch, sub, old, new):
    path = os.path.join(os.path.dirname(oracle.__file__), sub + ".py")
    src = open(path).read()
    if old is not None:
        assert src.count(old) == 1, f"mutation site not unique: {old!r}"
        src = src.replace(old, new)
    mod = types.ModuleType("oracle." + sub)
    mod.__file__ = path
    mod.__package__ = "oracle"
    exec(compile(src, path, "exec"), mod.__dict__)
    monkeypatch.setitem(sys.modules, "oracle." + sub, mod)
    monkeypatch.setattr(oracle, sub, mod, raising=False)
    return [_load_module(SUB_PINS[sub])]


PY_MUTATIONS = [
    # entry contexts (the serial scan's state at an offset)
    ("contexts", "context one byte late", "q = int(a.delta[q, w[p - 1]])", "q = int(a.delta[q, w[p]])"),
    ("contexts", "halting offset not a boundary", "ctx[s] = BOUNDARY           # s == con(w)", "pass"),
    ("contexts", "candidates without BOUNDARY", "return [BOUNDARY] + sorted(out)", "return sorted(out)"),
    ("contexts", "first accepting end in a chunk run",
     "last, kind = j, int(a.tau[q])\n    return last, kind",
     "last, kind = j, int(a.tau[q])\n            break\n    return last, kind"),
    ("contexts", "exit context from the chunk start",
     "_state_after(a, w, a.q0, pos, p1)), None\n        pos = e",
     "_state_after(a, w, a.q0, p0, p1)), None\n        pos = e"),
    ("contexts", "exit context not passed on", "toks, ctx, fail = chunk_run(a, w, p0, p1, ctx)",
     "toks, _, fail = chunk_run(a, w, p0, p1, ctx)"),
    # live sets (the failed-lookahead guard)
    ("live", "walk starts one byte late", "        j = k\n", "        j = k + 1\n"),
    ("live", "acceptance only at the end of the input", "hit = acc[cur]", "hit = acc[cur] & (j + 1 == n)"),
    ("live", "guard reads the next offset's set", "while j < n and live[j, q]:",
     "while j < n and live[min(j + 1, n), q]:"),
    ("live", "guarded scan ends every token at the first accept",
     "last, kind = j, int(a.tau[q])\n        if last is None:",
     "last, kind = j, int(a.tau[q])\n                break\n        if last is None:"),
    # two-byte split windows
    ("windows", "delta+ leaving Q+ counted as defined", "return t if t >= 0 and live[q] and live[t] else -1",
     "return t if t >= 0 else -1"),
    ("windows", "Z(a) without the states that start a token",
     "Z = {dplus(q, x) for q in states} - {-1}", "Z = {dplus(q, x) for q in states if q != a.q0} - {-1}"),
    ("windows", "delta+(q0, b) not required", "if dplus(a.q0, y) < 0:\n                continue", "pass"),
    ("windows", "window bytes transposed", "P[w[p - 1], w[p]]", "P[w[p], w[p - 1]]"),
    # the FP64 model
    ("model", "kernel flipped in the forward convolution", "hp[:, k:k + W], Wc[:, k, :])",
     "hp[:, K - 1 - k:K - 1 - k + W], Wc[:, k, :])"),
    ("model", "softmax gradient without the label term", "dz[np.arange(B), y] -= 1.0", "pass"),
    ("model", "sum instead of mean in the gradient", "dz /= B", "pass"),
    ("model", "hidden ReLU mask dropped", "da1 = (dz @ W2.T) * (a1 > 0)", "da1 = dz @ W2.T"),
    ("model", "embedding gradient with repeated bytes overwritten", "np.add.at(gemb, x, dh0)", "gemb[x] += dh0"),
    ("model", "window one byte late", "q = int(p) - W // 2 + k", "q = int(p) - W // 2 + k + 1"),
    ("model", "bfloat16 by truncation", "r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16", "r = (u >> 16) << 16"),
]


@pytest.mark.parametrize("sub", sorted(SUB_PINS))
def test_unmutated_submodule_passes_its_pins(monkeypatch, sub):
    mods = _swap_submodule(monkeypatch, sub, None, None)
    assert _failing_pins(mods) == []


@pytest.mark.parametrize("sub,name,old,new", PY_MUTATIONS, ids=[f"{m[0]}: {m[1]}" for m in PY_MUTATIONS])
def test_planted_mistake_in_a_python_oracle_fails_a_pin(monkeypatch, sub, name, old, new):
    mods = _swap_submodule(monkeypatch, sub, old, new)
    assert _failing_pins(mods, first=True), f"no pin catches: {sub}: {name}"
