#!/usr/bin/env python3
"""Generate regwin_dispatch.cuh: jump-table dispatch for the REGWIN kernel.

The REGWIN kernel adds win[o + q] (q < SPL) into the SPL sums of one DM trial,
where the offset o (0..31) is only known at run time but is the same for
every lane of the warp.  Register arrays cannot be indexed at run time, so
each offset needs its own straight-line code; a C++ switch over 32 cases is
compiled into a compare-and-branch tree, which measured ~5x slower than the
adds it guards.  This generator emits inline PTX that jumps once, through a
`brx.idx.uni` table, to the code for the offset.  It also emits the window
load: a fall-through chain entered at the number of extra samples the
channel needs, so exactly SPL + extra shared loads issue.

Run: python gen_regwin_dispatch.py > regwin_dispatch.cuh
"""
import sys

NOFF = 32            # offsets 0..31
SPLS = (11, 15)


def add_fn(spl: int, weighted: bool) -> str:
    nacc, nwin = spl, spl + NOFF - 1
    # operands: %0..%(spl-1) acc (in/out); %spl = o; then win[0..nwin-1]; then w
    o_idx = nacc
    w0 = nacc + 1
    wt = w0 + nwin
    lines = ["{", "ts: .branchtargets " + ", ".join(f"L{k}" for k in range(NOFF)) + ";",
             f"brx.idx.uni %{o_idx}, ts;"]
    for k in range(NOFF):
        body = []
        for q in range(spl):
            if weighted:
                body.append(f"fma.rn.f32 %{q}, %{w0 + k + q}, %{wt}, %{q};")
            else:
                body.append(f"add.rn.f32 %{q}, %{q}, %{w0 + k + q};")
        tail = " bra.uni LE;" if k != NOFF - 1 else ""
        lines.append(f"L{k}: " + " ".join(body) + tail)
    lines.append("LE:")
    lines.append("}")
    asm = "\\n\\t".join(lines)
    outs = ", ".join(f'"+f"(acc[{q}])' for q in range(nacc))
    ins = [f'"r"(o)'] + [f'"f"(win[{k}])' for k in range(nwin)]
    if weighted:
        ins.append('"f"(w)')
    name = "fma" if weighted else "add"
    wparam = ", float w" if weighted else ""
    return (f"  static __device__ __forceinline__ void {name}(float (&acc)[{spl}], const float (&win)[{nwin}], "
            f"uint32_t o{wparam}) {{\n"
            f"    asm(\"{asm}\"\n        : {outs}\n        : {', '.join(ins)});\n  }}\n")


def load_fn(spl: int) -> str:
    nwin = spl + NOFF - 1
    # operands: %0..%(nwin-1) win (in/out); %nwin = extra; %nwin+1 = shared address
    e_idx, a_idx = nwin, nwin + 1
    lines = ["{", "ts: .branchtargets " + ", ".join(f"L{k}" for k in range(NOFF)) + ";",
             f"brx.idx.uni %{e_idx}, ts;"]
    for k in range(NOFF - 1, 0, -1):
        r = spl + k - 1
        lines.append(f"L{k}: ld.shared.f32 %{r}, [%{a_idx}+{4 * r}];")
    base = " ".join(f"ld.shared.f32 %{q}, [%{a_idx}+{4 * q}];" for q in range(spl))
    lines.append(f"L0: {base}")
    lines.append("}")
    asm = "\\n\\t".join(lines)
    outs = ", ".join(f'"+f"(win[{k}])' for k in range(nwin))
    return (f"  static __device__ __forceinline__ void load(float (&win)[{nwin}], uint32_t extra, uint32_t saddr) {{\n"
            f"    asm volatile(\"{asm}\"\n        : {outs}\n        : \"r\"(extra), \"r\"(saddr) : \"memory\");\n  }}\n")


def main():
    out = ["// Generated by gen_regwin_dispatch.py -- do not edit by hand.",
           "// Jump-table dispatch (brx.idx.uni) for the REGWIN forward kernel:",
           "//   add/fma: acc[q] += win[o + q] (* w), q < SPL, o in [0, 31] warp-uniform;",
           "//   load:    win[0 .. SPL + extra) <- shared[saddr ...], extra in [0, 31] warp-uniform.",
           "#pragma once", "#include <cstdint>", "", "namespace dd {", "",
           f"constexpr int kRwDispatchOffsets = {NOFF};", "",
           "template <int SPL>", "struct RwDispatch;", ""]
    for spl in SPLS:
        out.append(f"template <>\nstruct RwDispatch<{spl}> {{")
        out.append(add_fn(spl, False))
        out.append(add_fn(spl, True))
        out.append(load_fn(spl))
        out.append("};\n")
    out.append("}  // namespace dd")
    sys.stdout.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
