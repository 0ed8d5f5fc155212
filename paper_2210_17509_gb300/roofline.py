"""Roofline bookkeeping for the benchmark: algorithmic work per cell and peaks.

Algorithmic FP64 operations of the fused RHS kernel per interior cell, counted
by hand from the 3+1 formulas the kernel evaluates (add, sub, mul = 1, fused
multiply-add = 2, divide and square root = 1, min/max = 1), with the three
faces per cell counted once (tile-boundary recomputation is not algorithmic):

  WENO5 reconstruction of one value            69   (candidates 16, indicators 36, weights 17)
  face metric (mean of 2 cells, sqrt(gamma), gamma^dd)   42
  one side of a face (cons, flux, signal speeds) 160
  HLLE combination                              65
  per face (WENO5): 16 * 69 + 42 + 2 * 160 + 65 = 1531
  flux divergence                               72
  source terms (FD4 metric derivatives, T^{mu nu}, Eq. 13 in 3+1 form)  666
  stage epilogue                                40
  cell total (curved, WENO5): 3 * 1531 + 72 + 666 + 40 = 5371

The FP64 RHS of the cached paths runs in three passes: rhs_states_kernel
(WENO5 reconstruction, both states of every cell per direction: 3 * 16 * 69
flops per cell counted per face as below), rhs_face_kernel (face metric,
side states and HLLE of every face once) and rhs_div_kernel (divergence,
sources, epilogue: 72 + 666 + 40).  The unit the benchmark times is that
triple (one grmhd_rhs_cached call); the two first passes together do the
3 * 1531 flops of the faces.

Algorithmic HBM bytes per interior cell of the triple (FP64, static metric,
geometry cache): prim 8 x 8 B + geometry cache 63 x 8 B read (the face pass
reads the half-metric and face entries, the per-cell pass the rest), rhs
8 x 8 B written = 632 B, plus the face buffer, 24 x 8 B written and read
back = 384 B, and the state buffer, 48 x 8 B written and read back = 768 B:
1784 B (the uncached single-pass grmhd_rhs reads the 10 metric entries
instead of the cache and has no buffers: 208 B).

Measured DRAM traffic of the triple (ncu, dram__bytes_read.sum +
dram__bytes_write.sum, all three kernels) for the 96^3 block (884,736
cells, capture in profiles/rhs_three_pass_fp64_cached_weno5_curved_96cube.md):
405.4 + 754.5 + 786.7 MB = 1946.6 MB, 2200 B per cell; traffic grows with
the cell count, so a launch on n^3 cells is 2200 n^3 B.

Peaks: HBM copy bandwidth from the generated MEASURED_PEAKS.json; the
FP64 FMA peak was measured on this GPU model with ``python -m
paper_2210_17509_gb300.peaks`` at the 2070 MHz SM clock the benchmark runs
at: 1.256 TFLOP/s (FMA = 2 flops), i.e. 2 FP64 FMA per SM per clock on 152
SMs (1.20 TFLOP/s in an earlier run at 2.0 GHz).
"""
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FLOPS_PER_CELL_RHS_CURVED_WENO5 = 5371
BYTES_PER_CELL_RHS_CURVED = 632 + 384 + 768
TRAFFIC_PER_CELL_MEASURED = (405.4e6 + 754.5e6 + 786.7e6) / 884736  # 2200 B per cell
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
    flops = FLOPS_PER_CELL_RHS_CURVED_WENO5 * ncells
    achieved = flops / (ms_per_launch * 1e-3) / 1e12
    hbm, src = hbm_peak_gbs()
    if traffic == "measured":
        traffic = None if TRAFFIC_PER_CELL_MEASURED is None else TRAFFIC_PER_CELL_MEASURED * ncells
    gbs = BYTES_PER_CELL_RHS_CURVED * ncells / (ms_per_launch * 1e-3) / 1e9
    return {
        "bound": "alu",
        "kernel": "rhs_states_kernel + rhs_face_kernel + rhs_div_kernel<double, WENO5, curved, geometry cache> "
                  "(grmhd_rhs_cached, FP64)",
        "achieved": achieved, "peak": FP64_PEAK_TFLOPS_MEASURED, "unit": "TFLOP/s",
        "frac": achieved / FP64_PEAK_TFLOPS_MEASURED, "traffic": traffic,
        "peak_source": "measured FP64 FMA probe (python -m paper_2210_17509_gb300.peaks)",
        "ms_per_launch": ms_per_launch, "flops_per_cell": FLOPS_PER_CELL_RHS_CURVED_WENO5,
        "hbm_context": {"achieved_gbs": gbs, "peak_gbs": hbm, "peak_source": src, "frac": gbs / hbm,
                        "bytes_per_cell": BYTES_PER_CELL_RHS_CURVED},
    }
