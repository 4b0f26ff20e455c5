#!/usr/bin/env python3
"""Writes fwd_u8_dispatch.inc: the per-channel DM-offset dispatch of fwd_u8.cu.

For a tile of DR DMs per lane, the macro DD_U8_CHANNEL_<DR>(A, R, IX) adds,
for every DM i < DR, the 20-word register slice R[IX[i] .. IX[i] + 20) of the
lane's window into the accumulators A[i][0 .. 20), with IX[i] in [0, 16).

It is one inline-PTX block laid out as a chain of indexed branches: block
(i, k) does the 20 adds of DM i at offset k and then jumps straight to block
(i + 1, IX[i + 1]) with a warp-uniform brx.idx, so each DM costs one indexed
branch and no join branch.  Writing the dispatch in PTX keeps it that way; a
C++ switch over the same cases became a chain of compares and branches.

Run from this directory:  python gen_u8_dispatch.py  (regenerates the .inc).
"""
import os

H, CASES, WIN = 20, 16, 36
SHAPES = (4, 6, 8)


def macro(dr):
    nacc = dr * H
    lines = ['"{\\n\\t"']
    for i in range(dr):
        targets = ", ".join(f"ddu8c{dr}_d{i}_k{k}" for k in range(CASES))
        lines.append(f'"ddu8c{dr}_t{i}: .branchtargets {targets};\\n\\t"')
    lines.append(f'"brx.idx.uni %{nacc + WIN}, ddu8c{dr}_t0;\\n\\t"')
    for i in range(dr):
        for k in range(CASES):
            lines.append(f'"ddu8c{dr}_d{i}_k{k}:\\n\\t"')
            for j in range(H):
                lines.append(f'"add.u32 %{i * H + j}, %{i * H + j}, %{nacc + k + j};\\n\\t"')
            if i + 1 < dr:
                lines.append(f'"brx.idx.uni %{nacc + WIN + i + 1}, ddu8c{dr}_t{i + 1};\\n\\t"')
            elif k != CASES - 1:
                lines.append(f'"bra.uni ddu8c{dr}_end;\\n\\t"')
    lines.append(f'"ddu8c{dr}_end:\\n\\t}}"')
    outs = ", ".join(f'"+r"(A[{i}][{j}])' for i in range(dr) for j in range(H))
    ins = ", ".join(f'"r"(R[{j}])' for j in range(WIN))
    ins += ", " + ", ".join(f'"r"(IX[{i}])' for i in range(dr))
    out = [f"#define DD_U8_CHANNEL_{dr}(A, R, IX) \\", "  asm volatile( \\"]
    out += [f"      {ln} \\" for ln in lines]
    out.append(f"      : {outs} \\")
    out.append(f"      : {ins})")
    return out


def main():
    out = ["// Generated by gen_u8_dispatch.py; do not edit.", "#pragma once", "// NOLINTBEGIN"]
    for dr in SHAPES:
        out += macro(dr)
        out.append("")
    out.append("// NOLINTEND")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fwd_u8_dispatch.inc")
    with open(path, "w") as fh:
        fh.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
