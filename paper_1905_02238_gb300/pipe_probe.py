"""Runs the pipe-rate probe (csrc/pipe_probe.cu): issue rates of ex2 / rcp on the SFU and of FP32
and packed-FP32 FMAs per SM per clock on this GPU, the figures behind the exact kernel's roofline.

    python -m paper_1905_02238_gb300.pipe_probe
"""
from __future__ import annotations

import subprocess
import sys

from . import build


def main() -> int:
    return subprocess.run([build.build_probe()]).returncode


if __name__ == "__main__":
    sys.exit(main())
