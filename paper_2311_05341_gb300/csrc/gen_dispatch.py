#!/usr/bin/env python3
"""Generates the per-channel DM-offset dispatch used by fwd_tiled.cu.

For a register tile of DR DMs per lane, DD_TILE_CHANNEL_<OP>_<DR>(A, R, IX)
adds, for every DM i < DR, the 20-word register slice R[IX[i] .. IX[i] + 20)
of the lane's 36-word window into the accumulators A[i][0 .. 20), with IX[i]
in [0, 16).  OP is U32 (packed 16-bit lanes or uint16 samples in 32-bit words)
or F32 (float samples).

Each macro is one inline-PTX block laid out as a chain of indexed branches:
block (i, k) does the 20 adds of DM i at offset k and then jumps straight to
block (i + 1, IX[i + 1]) with a warp-uniform brx.idx, so each DM costs one
indexed branch and no join branch.  (A C++ switch over the same cases became
a chain of compares and branches.)  The build writes the result into the
build directory; nothing generated is committed.
"""
import os
import sys

H, CASES, WIN = 20, 16, 36
SHAPES = (1, 2, 4, 6, 8)
OPS = {"U32": ("add.u32", "r"), "F32": ("add.f32", "f")}


def macro(op, dr):
    instr, cons = OPS[op]
    tag = f"ddt{op.lower()}{dr}"
    nacc = dr * H
    lines = ['"{\\n\\t"']
    for i in range(dr):
        targets = ", ".join(f"{tag}_d{i}_k{k}" for k in range(CASES))
        lines.append(f'"{tag}_t{i}: .branchtargets {targets};\\n\\t"')
    lines.append(f'"brx.idx.uni %{nacc + WIN}, {tag}_t0;\\n\\t"')
    for i in range(dr):
        for k in range(CASES):
            lines.append(f'"{tag}_d{i}_k{k}:\\n\\t"')
            for j in range(H):
                lines.append(f'"{instr} %{i * H + j}, %{i * H + j}, %{nacc + k + j};\\n\\t"')
            if i + 1 < dr:
                lines.append(f'"brx.idx.uni %{nacc + WIN + i + 1}, {tag}_t{i + 1};\\n\\t"')
            elif k != CASES - 1:
                lines.append(f'"bra.uni {tag}_end;\\n\\t"')
    lines.append(f'"{tag}_end:\\n\\t}}"')
    outs = ", ".join(f'"+{cons}"(A[{i}][{j}])' for i in range(dr) for j in range(H))
    ins = ", ".join(f'"{cons}"(R[{j}])' for j in range(WIN))
    ins += ", " + ", ".join(f'"r"(IX[{i}])' for i in range(dr))
    out = [f"#define DD_TILE_CHANNEL_{op}_{dr}(A, R, IX) \\", "  asm volatile( \\"]
    out += [f"      {ln} \\" for ln in lines]
    out.append(f"      : {outs} \\")
    out.append(f"      : {ins})")
    return out


PATTERN_H = (15, 17, 19, 21, 23, 25)  # odd window words per lane of the pattern tiles
PATTERN_DR = 4


def pattern_macro(op, h):
    """DD_PAT_CHANNEL_<OP>_<H>(A, R, IX): 4 DMs of one lane, one indexed branch.

    R holds the lane's h + 6 window words, loaded before the branch; block IX
    (a pattern with base increment a <= 1, see _pattern_offsets) adds
    R[o_i .. o_i + h) into A[i][0 .. h) for the four DMs i.
    """
    instr, cons = OPS[op]
    tag = f"ddp{op.lower()}{h}"
    nacc = PATTERN_DR * h
    win = h + 2 * (PATTERN_DR - 1)
    npat = 16
    lines = ['"{\\n\\t"']
    targets = ", ".join(f"{tag}_p{p}" for p in range(npat))
    lines.append(f'"{tag}_t: .branchtargets {targets};\\n\\t"')
    lines.append(f'"brx.idx.uni %{nacc + win}, {tag}_t;\\n\\t"')
    for p in range(npat):
        offs = _pattern_offsets(p)
        lines.append(f'"{tag}_p{p}:\\n\\t"')
        for i in range(PATTERN_DR):
            for j in range(h):
                lines.append(f'"{instr} %{i * h + j}, %{i * h + j}, %{nacc + offs[i] + j};\\n\\t"')
        if p != npat - 1:
            lines.append(f'"bra.uni {tag}_end;\\n\\t"')
    lines.append(f'"{tag}_end:\\n\\t}}"')
    outs = ", ".join(f'"+{cons}"(A[{i}][{j}])' for i in range(PATTERN_DR) for j in range(h))
    ins = ", ".join(f'"{cons}"(R[{j}])' for j in range(win)) + ', "r"(IX)'
    out = [f"#define DD_PAT_CHANNEL_{op}_{h}(A, R, IX) \\", "  asm volatile( \\"]
    out += [f"      {ln} \\" for ln in lines]
    out.append(f"      : {outs} \\")
    out.append(f"      : {ins})")
    return out


PAIR_H = (15, 17, 19, 21, 23, 25)  # window words per lane of the channel-pair pattern tiles
# In-block loads run this many words ahead of the adds that consume them, so a
# word's register dies after its last use (None: all loads first).  Integer
# blocks: 8 (the packed uint8 pair tile ran 1.7 % faster than with 4; the
# plain one and the float blocks were unchanged).
LOAD_AHEAD = {"U32": 8, "F32": 4, "F2": 4}
PACKED_PAIR_AHEAD = 7


# Channel pairs whose two window words are summed once per word (t_k + u_k)
# before the four DMs add that sum: (h + o_3) + 4 h adds per pair instead of
# 8 h.  Float pairs only (integer pairs already add both channels in one
# three-input add per accumulator).
PRESUM = {"F2"}
LOAD = {"U32": ("ld.shared.b32", ".b32"), "F32": ("ld.shared.f32", ".f32"),
        "F2": ("ld.shared.b64", ".b64")}
# Float pairs: 64-bit window words of two floats (samples u and u + 32 H),
# added two at a time.
OPS_F2 = ("add.rn.f32x2", "l")
WORD_BYTES = {"U32": 4, "F32": 4, "F2": 8}
F2_H = (11, 13)  # window words per lane of the float-pair pattern tiles


PATTERNS = 32  # 8 base increments a = 0..3 x the 8 patterns of +0/+1 on top


def _pattern_offsets(p):
    """Offsets of a warp's 4 DMs for pattern p = 8 a + b: increment k is
    a + bit k of b."""
    a, b = divmod(p, 8)
    inc = [a + ((b >> k) & 1) for k in range(3)]
    return [0, inc[0], inc[0] + inc[1], inc[0] + inc[1] + inc[2]]


def pattern_load_macro(op, h, pair, ahead=None, suffix=""):
    """Pattern blocks that load their own window words.

    DD_PATL_CHANNEL_<OP>_<H>(A, S, IX) and, for two channels of one pattern,
    DD_PATL2_CHANNEL_U32_<H>(A, S, S2, IX): S (S2) is the shared-memory
    address of the lane's window.  Block p loads only the h + o_3 words its
    offsets (0, o_1, o_2, o_3) touch, then DM i adds words o_i .. o_i + h
    into A[i][0 .. h).
    """
    ahead_override = ahead
    instr, cons = OPS_F2 if op == "F2" else OPS[op]
    ld, ty = LOAD[op]
    wb = WORD_BYTES[op]
    tag = f"ddl{('q' if op == 'U32' else 'q' + op.lower()) if pair else op.lower()}{h}{suffix.lower()}"
    nacc = PATTERN_DR * h
    win = h + max(_pattern_offsets(p)[3] for p in range(PATTERNS))
    s1 = nacc
    s2 = nacc + 1
    ix = nacc + (2 if pair else 1)
    regs = f".reg {ty} t<{win}>;" + (f" .reg {ty} u<{win}>;" if pair else "")
    lines = ['"{\\n\\t"', f'"{regs}\\n\\t"']
    targets = ", ".join(f"{tag}_p{p}" for p in range(PATTERNS))
    lines.append(f'"{tag}_t: .branchtargets {targets};\\n\\t"')
    lines.append(f'"brx.idx.uni %{ix}, {tag}_t;\\n\\t"')
    for p in range(PATTERNS):
        offs = _pattern_offsets(p)
        n = h + offs[3]
        lines.append(f'"{tag}_p{p}:\\n\\t"')

        def load(k):
            lines.append(f'"{ld} t{k}, [%{s1}+{wb * k}];\\n\\t"')
            if pair:
                lines.append(f'"{ld} u{k}, [%{s2}+{wb * k}];\\n\\t"')

        presum = pair and op in PRESUM

        def add(i, j):
            a = i * h + j
            lines.append(f'"{instr} %{a}, %{a}, t{offs[i] + j};\\n\\t"')
            if pair and not presum:
                lines.append(f'"{instr} %{a}, %{a}, u{offs[i] + j};\\n\\t"')

        ahead = LOAD_AHEAD[op] if ahead_override is None else ahead_override
        assert ahead is not None or not presum
        if ahead is None:
            for k in range(n):
                load(k)
            for i in range(PATTERN_DR):
                for j in range(h):
                    add(i, j)
        else:
            for k in range(min(ahead, n)):
                load(k)
            for k in range(n):  # adds consuming word k, then the next load
                if presum:  # every word k < h + o_3 is read by some DM
                    lines.append(f'"{instr} t{k}, t{k}, u{k};\\n\\t"')
                for i in range(PATTERN_DR):
                    if 0 <= k - offs[i] < h:
                        add(i, k - offs[i])
                if k + ahead < n:
                    load(k + ahead)
        if p != PATTERNS - 1:
            lines.append(f'"bra.uni {tag}_end;\\n\\t"')
    lines.append(f'"{tag}_end:\\n\\t}}"')
    outs = ", ".join(f'"+{cons}"(A[{i}][{j}])' for i in range(PATTERN_DR) for j in range(h))
    ins = '"r"(S), "r"(S2), "r"(IX)' if pair else '"r"(S), "r"(IX)'
    name = (f"DD_PATL2_CHANNEL_{op}{suffix}_{h}(A, S, S2, IX)" if pair
            else f"DD_PATL_CHANNEL_{op}{suffix}_{h}(A, S, IX)")
    out = [f"#define {name} \\", "  asm volatile( \\"]
    out += [f"      {ln} \\" for ln in lines]
    out.append(f"      : {outs} \\")
    out.append(f"      : {ins} \\")
    out.append('      : "memory")')
    return out


def generate(path):
    out = ["// Generated by gen_dispatch.py at build time.", "#pragma once"]
    for op in OPS:
        for dr in SHAPES:
            out += macro(op, dr)
            out.append("")
        for h in PATTERN_H:
            out += pattern_macro(op, h)
            out.append("")
    for h in PATTERN_H:
        for op in OPS:
            out += pattern_load_macro(op, h, False)
            out.append("")
    for h in PAIR_H:
        out += pattern_load_macro("U32", h, True)
        out.append("")
        # Packed copies (kU8P): loads 7 words ahead (0.8 % faster than 8 on
        # the paper uint8 plan with phased widening; the other kinds keep 8).
        out += pattern_load_macro("U32", h, True, ahead=PACKED_PAIR_AHEAD, suffix="P")
        out.append("")
    for h in F2_H:
        out += pattern_load_macro("F2", h, False)
        out.append("")
        out += pattern_load_macro("F2", h, True)
        out.append("")
    text = "\n".join(out) + "\n"
    os.makedirs(os.path.dirname(path), exist_ok=True)
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, "w") as fh:
            fh.write(text)
    return path


if __name__ == "__main__":
    print(generate(sys.argv[1] if len(sys.argv) > 1 else "fwd_tiled_dispatch.inc"))
