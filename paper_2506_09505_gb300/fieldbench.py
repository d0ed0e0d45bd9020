"""Per-operation throughput of the GPU Goldilocks basic functions (the
counterparts of the paper's Table 1, measured like its Sec. 4.3 study but
with CUDA events and clock64 instead of perf counters).

    python -m paper_2506_09505_gb300.fieldbench
"""
import json
import sys

from . import field_bench, init, load

OPS = ["add", "sub", "reduce", "sqr", "mul", "mul_small", "sbox", "dot12",
       "pipe_imad", "pipe_imad_wide", "pipe_iadd"]
LAT_OPS = ["lat_mul", "lat_sbox", "lat_dot12", "lat_perm", "lat_perm_wide"]
# 32-bit multiply results per operation (IMAD.WIDE counts 2)
MUL_RESULTS = {"add": 0, "sub": 0, "reduce": 0, "sqr": 6, "mul": 8, "mul_small": 4, "sbox": 28, "dot12": 96,
               "pipe_imad": 1, "pipe_imad_wide": 2, "pipe_iadd": 0}


def main(argv=None):
    load(build_if_missing=True)
    init(0)
    rows = []
    for op in OPS:
        rate, per_clk = field_bench(op)
        rows.append({"op": op, "G_per_s": rate / 1e9, "per_sm_clock": per_clk,
                     "mul32_results_per_sm_clock": per_clk * MUL_RESULTS[op]})
    lat = []
    for op in LAT_OPS:
        rate, cycles = field_bench(op)
        lat.append({"op": op, "cycles": cycles, "per_s": rate})
    if argv and "--json" in argv:
        print(json.dumps({"throughput": rows, "latency": lat}))
    else:
        print(f"{'op':10s} {'G/s':>9s} {'per SM clk':>11s} {'mul32 res/clk/SM':>17s}")
        for r in rows:
            print(f"{r['op']:10s} {r['G_per_s']:9.2f} {r['per_sm_clock']:11.3f} {r['mul32_results_per_sm_clock']:17.1f}")
        print()
        print(f"{'latency (one warp, dependent chain)':36s} {'cycles':>9s}")
        for r in lat:
            print(f"{r['op']:36s} {r['cycles']:9.1f}")
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
