"""Mutation check of the oracle's pins: plausible mistakes are planted in copies of
oracle/ipg_oracle.c (a dropped term, a wrong comparison or index, a transposed
argument, a wrong combine), each copy is compiled on the CPU, and the CPU pin suites
(closed forms, library routines, hand-worked examples, random-graph properties) are run
against it through IPG_ORACLE_LIB.  Every mutant must fail at least one pin; the
unmodified source, built the same way, must pass them all."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ipg_oracle.c")
PIN_SUITES = ["tests/test_oracle_pins.py", "tests/test_oracle_pins_combiner.py", "tests/test_golden.py",
              "tests/test_oracle_properties.py"]

# (name, text in ipg_oracle.c, replacement, which occurrence (0-based), occurrences expected)
MUTANTS = [
    ("pagerank: base term not divided by N", "rank[v] = 0.15 / N + 0.85", "rank[v] = 0.15 + 0.85", 0, 1),
    ("pagerank: damping factors swapped", "rank[v] = 0.15 / N + 0.85", "rank[v] = 0.85 / N + 0.15", 0, 1),
    ("pagerank: message not divided by the out-degree", "double m = rank[v] / (double)outdeg;",
     "double m = rank[v];", 0, 1),
    ("pagerank: message from the receiver's rank", "double m = rank[v] / (double)outdeg;",
     "double m = rank[u] / (double)outdeg;", 0, 1),
    ("pagerank: initial rank 1", "rank[v] = 1.0 / N;", "rank[v] = 1.0;", 0, 1),
    ("hashmin: adopts larger labels", "changed = mb.msg[v] < label[v];", "changed = mb.msg[v] > label[v];", 0, 1),
    ("hashmin: senders and receivers transposed in the stats",
     "record(st, cap, s, active, senders, sent, receivers);",
     "record(st, cap, s, active, receivers, sent, senders);", 0, 4),
    ("min combiner keeps the maximum", "if (msg < mb->msg_next[dst]) mb->msg_next[dst] = msg;",
     "if (msg > mb->msg_next[dst]) mb->msg_next[dst] = msg;", 0, 1),
    ("receivers counted as every vertex", "for (uint32_t v = 0; v < n; ++v) r += mb->has[v];",
     "for (uint32_t v = 0; v < n; ++v) r += 1;", 0, 1),
    ("sssp: edge weights ignored", "uint64_t len = w ? (uint64_t)w[e] : 1u;", "uint64_t len = 1u;", 0, 2),
    ("sssp: active count not carried to the next superstep", "active = receivers;", "active = n;", 1, 4),
    ("sssp: source starts at distance 1", "cand = (s == 0) ? (v == source ? 0u : ORC_INF) : mb.msg[v];",
     "cand = (s == 0) ? (v == source ? 1u : ORC_INF) : mb.msg[v];", 0, 1),
    ("tree: a tie goes to the larger parent", "return x.b <= y.b ? x : y;", "return x.b >= y.b ? x : y;", 0, 1),
    ("tree: sends on a parent change too", "if (!dist_dropped) continue;", "", 0, 1),
    ("path counts: maximum instead of sum", "orc_msg r = {x.a, x.b + y.b};",
     "orc_msg r = {x.a, x.b > y.b ? x.b : y.b};", 0, 1),
    ("path counts: level not advanced", "orc_msg m = {(uint64_t)level[v] + 1, paths[v]};",
     "orc_msg m = {(uint64_t)level[v], paths[v]};", 0, 1),
    ("combine: or instead of exclusive or", "orc_msg r = {(uint32_t)(x.a ^ y.a), 0};",
     "orc_msg r = {(uint32_t)(x.a | y.a), 0};", 0, 1),
    ("combine: 64-bit minimum keeps the maximum", "return x.a <= y.a ? x : y;", "return x.a >= y.a ? x : y;", 0, 1),
    ("min mailbox keeps only the first message", "if (msg < mb->msg_next[dst]) mb->msg_next[dst] = msg;", ";",
     0, 1),
    ("sssp: the final superstep not counted", "        s++;\n        if (sent == 0) break;",
     "        if (sent == 0) break;\n        s++;", 1, 4),
    ("pagerank: one update too few", "for (s = 0; s <= updates; ++s) {", "for (s = 0; s + 1 <= updates; ++s) {",
     0, 1),
    ("hashmin: labels start at 0", "label[v] = v;", "label[v] = 0;", 0, 1),
]


def _mutate(text, old, new, which, expected):
    assert text.count(old) == expected, (old, text.count(old))
    at = -1
    for _ in range(which + 1):
        at = text.index(old, at + 1)
    return text[:at] + new + text[at + len(old):]


def _build(tmp, name, text):
    c = os.path.join(tmp, name + ".c")
    so = os.path.join(tmp, name + ".so")
    with open(c, "w") as f:
        f.write(text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", c, "-o", so])
    return so


def _run_pins(so):
    env = dict(os.environ, IPG_ORACLE_LIB=so)
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider"] + PIN_SUITES
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def test_pins_pass_on_the_unmodified_source(tmp_path):
    rc, out = _run_pins(_build(str(tmp_path), "control", open(SRC).read()))
    assert rc == 0, out


def test_every_planted_mistake_fails_a_pin(tmp_path):
    text = open(SRC).read()
    sos = [_build(str(tmp_path), "m%02d" % i, _mutate(text, old, new, which, exp))
           for i, (_, old, new, which, exp) in enumerate(MUTANTS)]
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(_run_pins, sos))
    survivors = [MUTANTS[i][0] for i, (rc, _) in enumerate(results) if rc == 0]
    assert not survivors, "mutants no pin catches: %s" % survivors
    errors = [(MUTANTS[i][0], out) for i, (rc, out) in enumerate(results) if rc not in (0, 1)]
    assert not errors, errors  # 1 = some test failed; anything else is a harness problem
