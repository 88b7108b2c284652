"""Planted mistakes in the oracle's Wa-Tor must fail its pins.

Each mutant is a copy of the oracle's C source with one plausible mistake in the
Wa-Tor rules (a swapped Philox stream id, a different counter layout, another
neighbour order or candidate map, a wrong breeding age, losers that do not age,
a wrong energy rule, a different initial draw), compiled on the CPU into a
temporary library.  The Wa-Tor pins of ``test_oracle_wator_brute`` and
``test_oracle_wator`` are then run with the mutant in place of ``orc_wator_run``;
at least one of them has to fail.  The real oracle is never modified.
"""
import ctypes
import inspect
import os
import subprocess

import numpy as np
import pytest

import oracle
import test_oracle_wator as pins_a
import test_oracle_wator_brute as pins_b

SRC = os.path.join(os.path.dirname(oracle.__file__), "dsoa_oracle.c")
HDR = os.path.join(os.path.dirname(oracle.__file__), "dsoa_oracle.h")

# (name, [(original text, mistaken text), ...]); every original must occur exactly once
MUTANTS = [
    ("fish draws on the shark stream",
     [("philox_w0(seed, t, f->cell, 1, 0)", "philox_w0(seed, t, f->cell, 2, 0)")]),
    ("shark draws on the fish stream",
     [("philox_w0(seed, t, s->cell, 2, 0)", "philox_w0(seed, t, s->cell, 1, 0)")]),
    ("stream ids swapped",
     [("philox_w0(seed, t, f->cell, 1, 0)", "philox_w0(seed, t, f->cell, 2, 0)"),
      ("philox_w0(seed, t, s->cell, 2, 0)", "philox_w0(seed, t, s->cell, 1, 0)")]),
    ("fish counter (cell, t) instead of (t, cell)",
     [("philox_w0(seed, t, f->cell, 1, 0)", "philox_w0(seed, f->cell, t, 1, 0)")]),
    ("shark counter stream in word 3",
     [("philox_w0(seed, t, s->cell, 2, 0)", "philox_w0(seed, t, s->cell, 0, 2)")]),
    ("E and W swapped",
     [("nb[1] = torus_nb(c, w, h, 1, 0);", "nb[1] = torus_nb(c, w, h, -1, 0);"),
      ("nb[3] = torus_nb(c, w, h, -1, 0);", "nb[3] = torus_nb(c, w, h, 1, 0);")]),
    ("N and S swapped",
     [("nb[0] = torus_nb(c, w, h, 0, -1);", "nb[0] = torus_nb(c, w, h, 0, 1);"),
      ("nb[2] = torus_nb(c, w, h, 0, 1);", "nb[2] = torus_nb(c, w, h, 0, -1);")]),
    ("order N, S, E, W",
     [("nb[1] = torus_nb(c, w, h, 1, 0);", "nb[1] = torus_nb(c, w, h, 0, 1);"),
      ("nb[2] = torus_nb(c, w, h, 0, 1);", "nb[2] = torus_nb(c, w, h, 1, 0);")]),
    ("fish candidate from the high bits",
     [("uint32_t tg = cand[u % k];\n                f->target", "uint32_t tg = cand[(u >> 16) % k];\n                f->target")]),
    ("shark candidate counted from the end",
     [("uint32_t tg = cand[u % k];\n                s->target", "uint32_t tg = cand[k - 1 - u % k];\n                s->target")]),
    ("fish breed at 4", [("#define WT_FISH_BREED 3u", "#define WT_FISH_BREED 4u")]),
    ("fish breed at 2", [("#define WT_FISH_BREED 3u", "#define WT_FISH_BREED 2u")]),
    ("sharks breed at 9", [("#define WT_SHARK_BREED 10u", "#define WT_SHARK_BREED 9u")]),
    ("sharks breed at 11", [("#define WT_SHARK_BREED 10u", "#define WT_SHARK_BREED 11u")]),
    ("losing fish do not age",
     [("f->age += 1;\n", ""),
      ("ev.fish_moves++;", "ev.fish_moves++; f->age += 1;")]),
    ("losing sharks do not age",
     [("s->age += 1;\n", ""),
      ("ev.shark_moves++;", "ev.shark_moves++; s->age += 1;")]),
    ("eating adds energy instead of refilling",
     [("s->energy = WT_SHARK_ENERGY;\n                } else",
       "s->energy += WT_SHARK_ENERGY;\n                } else")]),
    ("moving sharks keep their energy",
     [("} else {\n                    s->energy -= 1;\n                }",
       "} else {\n                }")]),
    ("newborn shark energy 2",
     [("ns->energy = WT_SHARK_ENERGY;", "ns->energy = 2;")]),
    ("initial draw on counter word 3",
     [("uint32_t u = philox_w0(seed, 0xFFFFFFFFu, c, 0, 0);\n            kind",
       "uint32_t u = philox_w0(seed, 0xFFFFFFFFu, 0, 0, c);\n            kind")]),
    ("initial fish and shark thresholds swapped",
     [("kind = u < WT_FISH_THR ? 1 : (u < WT_SHARK_THR ? 2 : 0);",
       "kind = u < WT_FISH_THR ? 2 : (u < WT_SHARK_THR ? 1 : 0);")]),
]


def _build(tmp_path, edits):
    src = open(SRC).read()
    for old, new in edits:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    c = tmp_path / "dsoa_oracle.c"
    c.write_text(src)
    (tmp_path / "dsoa_oracle.h").write_text(open(HDR).read())
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-std=c11", "-O1", "-ffp-contract=off", "-fPIC", "-shared",
                    "-w", "-o", str(so), str(c), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    P, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    lib.orc_wator_run.argtypes = [u32, u32, P, u64, u32, u32, u64, P, P]
    lib.orc_wator_run.restype = ctypes.c_int

    def run(w, h, steps, seed=0, init=None, t0=0, order_seed=0):
        ini = None if init is None else np.ascontiguousarray(np.asarray(init, np.uint8).reshape(-1))
        grid = np.zeros(w * h, np.uint8)
        stats = (oracle.WatorStep * max(steps, 1))()
        rc = lib.orc_wator_run(w, h, None if ini is None else ini.ctypes.data_as(P), seed,
                               steps, t0, order_seed, grid.ctypes.data_as(P),
                               ctypes.cast(stats, P))
        if rc != 0:
            raise RuntimeError("mutant oracle failed")
        rows = [{f: getattr(s, f) for f, _ in oracle.WatorStep._fields_} for s in stats[:steps]]
        return grid.reshape(h, w), rows
    return run


def _pin_calls():
    """Every Wa-Tor pin as a zero-argument call (parametrised pins expanded)."""
    calls = []
    for mod in (pins_b, pins_a):
        for name, fn in inspect.getmembers(mod, inspect.isfunction):
            if not name.startswith("test_") or fn.__module__ != mod.__name__:
                continue
            if "game_of_life" in name:
                continue
            marks = getattr(fn, "pytestmark", [])
            params = [m for m in marks if m.name == "parametrize"]
            if not params:
                calls.append((name, fn, {}))
                continue
            argnames, values = params[0].args[0], params[0].args[1]
            names = [a.strip() for a in argnames.split(",")]
            for v in values:
                v = v if isinstance(v, tuple) else (v,)
                calls.append((f"{name}{list(v)}", fn, dict(zip(names, v))))
    return calls


@pytest.mark.parametrize("name,edits", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_fails_a_pin(name, edits, tmp_path, monkeypatch):
    monkeypatch.setattr(oracle, "wator_run", _build(tmp_path, edits))
    caught = []
    for pin, fn, kw in _pin_calls():
        try:
            fn(**kw)
        except (AssertionError, RuntimeError):
            caught.append(pin)
    assert caught, f"no pin detects the mutant: {name}"


def test_unmutated_copy_passes_every_pin(tmp_path, monkeypatch):
    monkeypatch.setattr(oracle, "wator_run", _build(tmp_path, []))
    for _, fn, kw in _pin_calls():
        fn(**kw)
