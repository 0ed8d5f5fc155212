"""Roofline bookkeeping for the benchmark: work per cell and peaks.

Algorithmic FP64 operations of the RHS per interior cell come from
``flop_counts.json`` beside this file, which ``python -m oracle.flop_count``
writes: a counting scalar run through a plain 3+1 restatement of one cell's
RHS and stage update (WENO5 on 8 primitives to both sides of each face, face
metric, side states, signal speeds, HLLE, divergence with each face counted
once, Eq. 13 sources with 4th-order metric derivatives, stage combination;
+, -, *, /, sqrt, min, max = 1, a fused multiply-add = 2).  A test checks that
restatement against the oracle's RHS and the stored number against the
generator.

Executed FP64 operations per cell, for the second fraction: the ncu counts
of DADD, DMUL and DFMA thread instructions of the three FP64 RHS kernels
(rhs_states_kernel, rhs_face_kernel, rhs_div_kernel) at 96^3, as DADD + DMUL
+ 2 DFMA per interior cell.  The state pass works on the lines of cells -1 ..
n_d, so its count per interior cell falls with n as (n + 2) / n; at 256^3 it
is 0.8% below the 96^3 figure, which is used as it stands.

The algorithmic figure can exceed the FMA peak: the restatement forms every
face value on its own, where the kernels share work exactly (a cell's two
WENO5 states share their smoothness indicators and weights, neighbouring
cells of a line their first and second differences, the two sides of a face
1/alpha and one division), and it counts an add or a multiply as one flop,
as the hardware does, but two for each of its FMAs only where it writes one.
The FP64-pipe busy fractions (ncu) state the bound.

The FP64 RHS of the cached paths runs in three passes: rhs_states_kernel
(WENO5 states of every cell per direction), rhs_face_kernel (face metric,
side states and HLLE of every face once) and rhs_div_kernel (divergence,
sources, epilogue).  The unit the benchmark times is that triple (one
grmhd_rhs_cached call).

Algorithmic HBM bytes per interior cell of the triple (FP64, static metric,
geometry cache): prim 8 x 8 B + geometry cache 101 x 8 B read (the face
pass reads the face metric, 1/alpha, sqrt(gamma) and gamma^dd of the three
lower faces, 39 values; the per-cell pass the cell metric, the 30
derivatives and the 22 metric factors of the sources, 62 values), rhs 8 x 8
B written = 936 B, plus the face buffer, 24 x 8 B written and read back =
384 B, and the state buffer, 48 x 8 B written and read back = 768 B: 2088 B
(the uncached single-pass grmhd_rhs reads the 10 metric entries instead of
the cache and has no buffers: 208 B).

Measured DRAM traffic of the triple (ncu, dram__bytes_read.sum +
dram__bytes_write.sum, all three kernels) for the 96^3 block (884,736
cells): 462.1 + 829.7 + 949.7 MB = 2241.5 MB, 2534 B per cell (the per-cell
pass adds about 50 MB of register spills); traffic grows with the cell
count, so a launch on n^3 cells is about 2534 n^3 B.

Peaks: HBM copy bandwidth from the generated MEASURED_PEAKS.json; the
FP64 FMA peak was measured on this GPU model with ``python -m
paper_2210_17509_gb300.peaks`` at the 2070 MHz SM clock the benchmark runs
at: 1.256 TFLOP/s (FMA = 2 flops), i.e. 2 FP64 FMA per SM per clock on 152
SMs.
"""
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))

with open(os.path.join(HERE, "flop_counts.json")) as _f:
    FLOPS_PER_CELL_RHS_CURVED_WENO5 = int(json.load(_f)["rhs_curved_weno5_per_cell"])

# ncu thread-instruction counts per interior cell at 96^3 (DADD, DMUL, DFMA)
EXECUTED_FP64_PER_CELL = {"rhs_states_kernel": (233, 516, 551), "rhs_face_kernel": (76, 270, 370),
                          "rhs_div_kernel": (37, 66, 136)}
EXECUTED_FLOPS_PER_CELL = sum(a + m + 2 * f for a, m, f in EXECUTED_FP64_PER_CELL.values())
FP64_PIPE_BUSY = {"rhs_states_kernel": 0.863, "rhs_face_kernel": 0.896, "rhs_div_kernel": 0.807}
BYTES_PER_CELL_RHS_CURVED = 936 + 384 + 768
TRAFFIC_PER_CELL_MEASURED = (462.1e6 + 829.7e6 + 949.7e6) / 884736  # 2534 B per cell
FP64_PEAK_TFLOPS_MEASURED = 1.256
FP32_PEAK_TFLOPS_MEASURED = 78.5
HBM_FALLBACK_GBS = 6800.0


def hbm_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


def rhs_fp64_roofline(ncells: int, ms_per_launch: float, traffic="measured"):
    s = ms_per_launch * 1e-3
    achieved = FLOPS_PER_CELL_RHS_CURVED_WENO5 * ncells / s / 1e12
    executed = EXECUTED_FLOPS_PER_CELL * ncells / s / 1e12
    hbm, src = hbm_peak_gbs()
    if traffic == "measured":
        traffic = None if TRAFFIC_PER_CELL_MEASURED is None else TRAFFIC_PER_CELL_MEASURED * ncells
    gbs = BYTES_PER_CELL_RHS_CURVED * ncells / s / 1e9
    return {
        "bound": "alu",
        "kernel": "rhs_states_kernel + rhs_face_kernel + rhs_div_kernel<double, WENO5, curved, geometry cache> "
                  "(grmhd_rhs_cached, FP64)",
        "achieved": achieved, "peak": FP64_PEAK_TFLOPS_MEASURED, "unit": "TFLOP/s",
        "frac": achieved / FP64_PEAK_TFLOPS_MEASURED, "traffic": traffic,
        "peak_source": "measured FP64 FMA probe (python -m paper_2210_17509_gb300.peaks), of measured",
        "ms_per_launch": ms_per_launch, "flops_per_cell": FLOPS_PER_CELL_RHS_CURVED_WENO5,
        "flops_per_cell_source": "paper_2210_17509_gb300/flop_counts.json (python -m oracle.flop_count)",
        "executed": {"flops_per_cell": EXECUTED_FLOPS_PER_CELL, "achieved": executed,
                     "frac": executed / FP64_PEAK_TFLOPS_MEASURED,
                     "source": "ncu DADD + DMUL + 2 DFMA thread instructions per cell, 96^3"},
        "fp64_pipe_busy_ncu": FP64_PIPE_BUSY,
        "hbm_context": {"achieved_gbs": gbs, "peak_gbs": hbm, "peak_source": src, "frac": gbs / hbm,
                        "bytes_per_cell": BYTES_PER_CELL_RHS_CURVED},
    }
