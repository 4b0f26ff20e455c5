"""The generated shift-and-add blocks (csrc/gen_dispatch.py), executed
symbolically on the CPU.

Every block the generator writes is the inner step of Eq. 3 for one channel
(or two) and a few DMs: accumulator (i, j) of a lane adds window sample
s(c, d_i) + j.  The test runs the generated PTX text through a small
interpreter of the instruction forms the generator emits (labels,
`.branchtargets`, `brx.idx.uni`, `bra.uni`, `ld.shared`, `add`), with symbolic
values: a load gives the term (channel, word) and an add sums terms.  For
every branch index it checks that each accumulator ends as its start plus
exactly the window words the definition names, once each; that no register is
read before it is loaded or outside its declared array; that every word is
loaded once; and that the loads run the stated number of words ahead of the
adds.  A wrong offset, a dropped or doubled add, a load after its use or a
pre-sum applied twice fails here without a GPU.
"""
import importlib.util
import os
import re
from collections import Counter

import numpy as np
import pytest

_GEN = os.path.join(os.path.dirname(__file__), "..", "paper_2311_05341_gb300", "csrc",
                    "gen_dispatch.py")


@pytest.fixture(scope="module")
def gen():
    spec = importlib.util.spec_from_file_location("dd_gen_dispatch_test", _GEN)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _asm(lines):
    """The instructions of one generated macro, in order."""
    out = []
    for ln in lines:
        ln = ln.strip()
        if ln.endswith("\\"):
            ln = ln[:-1].rstrip()
        if not ln.startswith('"'):
            continue
        text = ln[1:ln.rindex('"')].replace("\\n", "\n").replace("\\t", "\t")
        out += [p.strip() for p in text.split("\n") if p.strip() and p.strip() not in "{}"]
    return out


def _n_operands(lines):
    return sum(len(re.findall(r'"\+?[rfl]"\(', ln)) for ln in lines
               if ln.strip().startswith(":"))


_LD = re.compile(r"ld\.shared\.(b32|f32|b64) ([tu])(\d+), \[%(\d+)\+(\d+)\];$")
_ADD = re.compile(r"add(?:\.\w+)+ (\S+), (\S+), (\S+);$")
_WB = {"b32": 4, "f32": 4, "b64": 8}


class _Run:
    """Executes one macro with asm operands `ops` (Counters for values,
    ints for branch indices, ('S', c) for the shared address of channel c)."""

    def __init__(self, instrs, ops):
        self.instrs = instrs
        self.ops = ops
        self.regs = {}
        self.decl = {}
        self.loads = Counter()
        self.hi = Counter()     # per channel: 1 + the highest word loaded so far
        self.reads = []         # (k, loaded so far) at each add reading t<k> / u<k>
        self.branches = 0       # indexed branches taken
        self.trace = []  # ('ld', channel, word) / ('add', dst) in order
        self.labels = {}
        self.tables = {}
        for k, ins in enumerate(instrs):
            m = re.match(r"(\w+): \.branchtargets (.*);$", ins)
            if m:
                self.tables[m.group(1)] = [t.strip() for t in m.group(2).split(",")]
            elif ins.endswith(":"):
                self.labels[ins[:-1]] = k

    def value(self, name):
        if name.startswith("%"):
            return self.ops[int(name[1:])]
        assert name in self.regs, f"{name} read before it is loaded"
        return self.regs[name]

    def run(self):
        pc = 0
        steps = 0
        while pc < len(self.instrs):
            steps += 1
            assert steps < 100000
            ins = self.instrs[pc]
            pc += 1
            for arr, n in re.findall(r"\.reg \.\w+ ([tu])<(\d+)>;", ins):
                self.decl[arr] = int(n)
            if ins.startswith(".reg") or ins.endswith(":") or ".branchtargets" in ins:
                continue
            m = re.match(r"brx\.idx\.uni %(\d+), (\w+);$", ins)
            if m:
                table = self.tables[m.group(2)]
                idx = self.ops[int(m.group(1))]
                assert 0 <= idx < len(table), "branch index outside its table"
                pc = self.labels[table[idx]]
                self.branches += 1
                continue
            m = re.match(r"bra\.uni (\w+);$", ins)
            if m:
                pc = self.labels[m.group(1)]
                continue
            m = _LD.match(ins)
            if m:
                ty, arr, k, base, off = m.groups()
                k, off = int(k), int(off)
                assert k < self.decl[arr], f"{arr}{k} outside .reg {arr}<{self.decl[arr]}>"
                kind, chan = self.ops[int(base)]
                assert kind == "S" and off % _WB[ty] == 0
                word = off // _WB[ty]
                self.regs[f"{arr}{k}"] = Counter({(chan, word): 1})
                self.loads[(chan, word)] += 1
                self.hi[chan] = max(self.hi[chan], word + 1)
                self.trace.append(("ld", chan, word))
                continue
            m = _ADD.match(ins)
            assert m, f"unexpected instruction {ins!r}"
            dst, a, b = m.groups()
            val = self.value(a) + self.value(b)
            if b[0] in "tu":
                self.reads.append((int(b[1:]), dict(self.hi)))
            if dst.startswith("%"):
                self.ops[int(dst[1:])] = val
            else:
                assert dst in self.regs
                self.regs[dst] = val
            self.trace.append(("add", dst))
        return self


def _acc(i, j):
    return Counter({("A", i, j): 1})


def _planner_patterns(amax):
    """(code, offsets) for every run of a warp's four DM shifts the planner
    accepts: increments i_k = s(c, d_k) - s(c, d_{k-1}) all a or a + 1 with
    a = min_k i_k <= amax, coded 8 a + sum_k (i_k - a) 2^(k-1) (plan.cpp,
    pattern_of).  DM k then reads window words s(c, d_k) - s(c, d_0) + j."""
    from itertools import product
    out = []
    for inc in product(range(amax + 2), repeat=3):
        a = min(inc)
        if a > amax or max(inc) - a > 1:
            continue
        code = 8 * a + sum((inc[k] - a) << k for k in range(3))
        offs = [0, inc[0], inc[0] + inc[1], inc[0] + inc[1] + inc[2]]
        out.append((code, offs))
    return out


@pytest.mark.parametrize("op,pair", [("U32", False), ("F32", False), ("U32", True),
                                     ("U32P", True), ("F2", False), ("F2", True)])
def test_pattern_load_blocks(gen, op, pair):
    """DD_PATL(2)_CHANNEL_*: the block of the planner's code for a warp's DM
    shifts adds words s(c, d_i) - s(c, d_0) + j of the lane's window (of both
    channels for pairs) into accumulator (i, j); each of the h + o_3 words is
    loaded once, the loads running `ahead` words in front of the adds."""
    base = "U32" if op == "U32P" else op
    hs = gen.F2_H if op == "F2" else gen.PAIR_H if pair else gen.PATTERN_H
    ahead = gen.PACKED_PAIR_AHEAD if op == "U32P" else gen.LOAD_AHEAD[base]
    presum = pair and base in gen.PRESUM
    chans = (1, 2) if pair else (1,)
    for h in hs:
        lines = (gen.pattern_load_macro(base, h, pair, ahead=gen.PACKED_PAIR_AHEAD, suffix="P")
                 if op == "U32P" else gen.pattern_load_macro(base, h, pair))
        instrs = _asm(lines)
        nacc = gen.PATTERN_DR * h
        assert _n_operands(lines) == nacc + len(chans) + 1
        pats = _planner_patterns(3)
        assert len(pats) == 28 and max(c for c, _ in pats) < gen.PATTERNS
        for p, offs in pats:
            ops = [_acc(i, j) for i in range(gen.PATTERN_DR) for j in range(h)]
            ops += [("S", c) for c in chans] + [p]
            r = _Run(instrs, ops).run()
            for i in range(gen.PATTERN_DR):
                for j in range(h):
                    want = _acc(i, j) + Counter({(c, offs[i] + j): 1 for c in chans})
                    assert r.ops[i * h + j] == want, (op, h, p, i, j)
            n = h + offs[3]
            assert r.loads == Counter({(c, k): 1 for c in chans for k in range(n)}), (op, h, p)
            # Loads issued before the first add: `ahead` words of each channel.
            first_add = next(k for k, t in enumerate(r.trace) if t[0] == "add")
            assert first_add == min(ahead, n) * len(chans), (op, h, p)
            # Every add that reads word k finds exactly words 0 .. k + ahead
            # of each channel loaded (all n at the end of the window).
            assert r.reads and all(hi == {c: min(n, k + ahead) for c in chans}
                                   for k, hi in r.reads), (op, h, p)
            if presum:  # one pre-sum per word, then four DMs' adds of it
                n_sum = sum(1 for t in r.trace if t[0] == "add" and not t[1].startswith("%"))
                assert n_sum == n
        # The codes the planner never emits still assemble: registers inside
        # their declared arrays, none read before its load.
        for p in sorted(set(range(gen.PATTERNS)) - {c for c, _ in pats}):
            ops = [_acc(i, j) for i in range(gen.PATTERN_DR) for j in range(h)]
            _Run(instrs, ops + [("S", c) for c in chans] + [p]).run()


@pytest.mark.parametrize("op", ["U32", "F32"])
def test_pattern_register_blocks(gen, op):
    """DD_PAT_CHANNEL_*: the block of the planner's code (base increment 0 or
    1) adds R[s(c, d_i) - s(c, d_0) + j] into accumulator (i, j)."""
    for h in gen.PATTERN_H:
        lines = gen.pattern_macro(op, h)
        instrs = _asm(lines)
        nacc = gen.PATTERN_DR * h
        win = h + 2 * (gen.PATTERN_DR - 1)
        assert _n_operands(lines) == nacc + win + 1
        for p, offs in _planner_patterns(1):
            assert p < 16 and offs[3] <= win - h
            ops = [_acc(i, j) for i in range(gen.PATTERN_DR) for j in range(h)]
            ops += [Counter({("R", k): 1}) for k in range(win)] + [p]
            r = _Run(instrs, ops).run()
            for i in range(gen.PATTERN_DR):
                for j in range(h):
                    assert r.ops[i * h + j] == _acc(i, j) + Counter({("R", offs[i] + j): 1})


@pytest.mark.parametrize("op", ["U32", "F32"])
def test_offset_register_blocks(gen, op):
    """DD_TILE_CHANNEL_*: DM i adds R[IX[i] + j] into accumulator (i, j), one
    indexed branch per DM, for seeded random and extreme offset vectors."""
    rng = np.random.default_rng(7)
    for dr in gen.SHAPES:
        lines = gen.macro(op, dr)
        instrs = _asm(lines)
        nacc = dr * gen.H
        assert _n_operands(lines) == nacc + gen.WIN + dr
        vecs = [[0] * dr, [gen.CASES - 1] * dr]
        vecs += [list(rng.integers(0, gen.CASES, dr)) for _ in range(24)]
        for ix in vecs:
            ops = [_acc(i, j) for i in range(dr) for j in range(gen.H)]
            ops += [Counter({("R", k): 1}) for k in range(gen.WIN)] + [int(v) for v in ix]
            r = _Run(instrs, ops).run()
            for i in range(dr):
                for j in range(gen.H):
                    assert r.ops[i * gen.H + j] == _acc(i, j) + Counter({("R", ix[i] + j): 1})
            assert r.branches == dr


def test_pattern_offsets_cover_every_increment_triple(gen):
    """Pattern p = 8 a + b: DM increments a + bit k of b.  The 32 patterns
    cover exactly the increment triples over 0..4 whose entries differ by at
    most one (the DM steps of a lane's four DMs differ by at most one sample);
    the all-equal triples 1..3 have two codes each."""
    from itertools import product
    seen = Counter()
    for p in range(gen.PATTERNS):
        o = gen._pattern_offsets(p)
        inc = tuple(o[k + 1] - o[k] for k in range(3))
        a, b = divmod(p, 8)
        assert inc == tuple(a + ((b >> k) & 1) for k in range(3))
        assert o[0] == 0
        seen[inc] += 1
    want = {t for t in product(range(5), repeat=3) if max(t) - min(t) <= 1}
    assert set(seen) == want and len(want) == 29
    assert sorted(t for t, n in seen.items() if n == 2) == [(1, 1, 1), (2, 2, 2), (3, 3, 3)]
