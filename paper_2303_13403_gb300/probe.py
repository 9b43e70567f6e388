"""Print the pipe micro-benchmarks of the current GPU as one JSON line.

  python -m paper_2303_13403_gb300.probe

FP64 FMA and FP64 tensor-core (DMMA) throughput, FP32 FMA throughput, the
latency of dependent FP64 FMA / divide / square root, and the cycles an FP64
warp instruction costs with 1, 8, 16 and 32 active lanes (pqmc_probe_pipes).
"""
import json

from . import pqmc


def main():
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(pqmc.probe_pipes()))


if __name__ == "__main__":
    main()
