"""Resource usage of the hot kernels (CPU: nvcc cross-compiles for sm_103a).

ptxas reports per kernel its registers, stack frame and spills.  The
reconstruction, splat, renderer stand-in, tensor-core convolution, weight
gradient, two-stage and variant kernels must not spill: a spill in one of
them turns register traffic into local-memory traffic in the hot loop.  The
persistent reconstruction kernel runs 512 threads per CTA, so it must fit
128 registers per thread.
"""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.join(ROOT, "paper_2602_08642_gb300"))
import build_lib  # noqa: E402

NO_SPILL = ["reconstruct_tma.cu", "render_splat.cu", "conv_tc.cu", "wgrad_tc.cu",
            "two_stage.cu", "variants.cu", "backward.cu", "reconstruct.cu"]


def _ptxas_report(src: str, out_dir: str) -> str:
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    obj = os.path.join(out_dir, os.path.basename(src) + ".o")
    cmd = [nvcc, *build_lib.ARCH, *build_lib.NVCC_FLAGS, "-Xptxas", "-v", "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout + r.stderr


def _kernels(report: str) -> dict:
    """name -> (registers, stack bytes, spill store bytes, spill load bytes)."""
    out, name = {}, None
    for line in report.splitlines():
        m = re.search(r"Function properties for (\S+)", line)
        if m:
            name = m.group(1)
            continue
        m = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads",
                      line)
        if m and name:
            out[name] = [None, int(m.group(1)), int(m.group(2)), int(m.group(3))]
            continue
        m = re.search(r"Used (\d+) registers", line)
        if m and name in out and out[name][0] is None:
            out[name][0] = int(m.group(1))
    return out


@pytest.fixture(scope="module")
def reports(tmp_path_factory):
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    d = str(tmp_path_factory.mktemp("ptxas"))
    srcs = [os.path.join(build_lib.CSRC, f) for f in NO_SPILL]
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        texts = list(ex.map(lambda s: _ptxas_report(s, d), srcs))
    return dict(zip(NO_SPILL, (_kernels(t) for t in texts)))


@pytest.mark.parametrize("src", NO_SPILL)
def test_hot_kernels_do_not_spill(reports, src):
    ks = reports[src]
    assert ks, f"no kernels reported for {src}"
    bad = {k: v for k, v in ks.items() if v[2] or v[3]}
    assert not bad, f"{src}: spilling functions {bad}"


def test_reconstruction_fits_512_threads(reports):
    recon = {k: v for k, v in reports["reconstruct_tma.cu"].items() if "recon_tma_kernel" in k}
    assert len(recon) >= 6  # the three levels, with and without the tone map
    for k, (regs, stack, _, _) in recon.items():
        assert regs is not None and regs <= 128, (k, regs)
        assert stack == 0, (k, stack)
