"""Build and run the FP64/FP32 arithmetic-peak probe on the current GPU.

    python -m paper_2210_17509_gb300.peaks            (needs nvcc and a GPU)
    python -m paper_2210_17509_gb300.peaks op-costs   (the FP64 operation-cost probe, for ncu)

Prints the probe's lines; the FP64 FMA rate it reports is the denominator the
benchmark uses for the FP64 ALU roofline (the generated peaks file holds
only HBM copy bandwidth and bf16 GEMM throughput).  The operation-cost probe
(op_costs.cu) runs one kernel per FP64 operation, whose ncu instruction
counts per element are that operation's cost.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def main():
    out_dir = os.path.join(ROOT, "_build")
    os.makedirs(out_dir, exist_ok=True)
    name = "op_costs" if sys.argv[1:] == ["op-costs"] else "fma_probe"
    exe = os.path.join(out_dir, name)
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-o", exe,
                    os.path.join(HERE, name + ".cu")], check=True)
    sys.exit(subprocess.run([exe]).returncode)


if __name__ == "__main__":
    main()
