"""Builds and runs csrc/peak_probe.cu (FP64/FP32 issue rates, HBM bandwidth,
a PRICE-shaped FP64 GEMV) and, with torch, times an FP64 DGEMM.

    python -m paper_1803_04378_gb300.peak_probe
"""
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = os.path.join(HERE, "_build", "peak_probe")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", out,
                    os.path.join(HERE, "csrc", "peak_probe.cu")], check=True)
    subprocess.run([out], check=True)
    import torch
    a = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    b = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    for _ in range(2):
        a @ b
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        a @ b
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 3
    print("torch DGEMM 4096^3: %.2f ms  %.2f TFLOP/s" % (ms, 2 * 4096 ** 3 / ms / 1e9))


if __name__ == "__main__":
    main()
