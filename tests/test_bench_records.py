"""The bench's DRAM-traffic records (profiles/ncu_traffic.txt): a record is
keyed by the hash of one kernel's device code, the header that defines it
and every header it includes; it stays valid through edits to other
kernels and to comments, and is dropped as soon as that code changes."""
import os
import shutil

import pytest

import bench

CSRC = os.path.join(bench.ROOT, "paper_1702_04458_b300", "csrc")


@pytest.fixture()
def tree(tmp_path, monkeypatch):
    """A copy of the kernel headers and an empty traffic file, as bench.ROOT."""
    csrc = tmp_path / "paper_1702_04458_b300" / "csrc"
    csrc.mkdir(parents=True)
    for name in os.listdir(CSRC):
        if name.endswith(".cuh"):
            shutil.copy(os.path.join(CSRC, name), csrc / name)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def _append(path, text):
    with open(path, "a", encoding="utf-8") as f:
        f.write(text)


def test_hash_covers_the_include_closure(tree):
    csrc = tree / "paper_1702_04458_b300" / "csrc"
    h0 = bench.kernel_source_hash("admm_ul_u32_tc5")
    # a header outside the tcgen05 kernel's closure, and a comment inside it
    _append(csrc / "dbp_tcdl.cuh", "\n__device__ int unrelated_edit;\n")
    _append(csrc / "dbp_tma.cuh", "\n// a comment only\n")
    assert bench.kernel_source_hash("admm_ul_u32_tc5") == h0
    # code in a header the kernel includes (dbp_tc32.cuh -> dbp_tma.cuh -> dbp_fused.cuh)
    _append(csrc / "dbp_fused.cuh", "\n__device__ int included_edit;\n")
    assert bench.kernel_source_hash("admm_ul_u32_tc5") != h0
    # the downlink kernel's closure does include dbp_tcdl.cuh
    h_dl = bench.kernel_source_hash("admm_dl")
    _append(csrc / "dbp_tcdl.cuh", "\n__device__ int second_edit;\n")
    assert bench.kernel_source_hash("admm_dl") != h_dl


def test_record_used_only_while_its_hash_matches(tree):
    src = bench.kernel_source_hash("admm_ul_u32_tc5")
    rec = tree / "profiles" / "ncu_traffic.txt"
    rec.write_text("# comment line\n"
                   f"#   kernel=admm_ul_u32_tc5 src={src} bytes_per_launch=7\n"      # superseded: skipped
                   f"kernel=admm_ul_u32_tc5 src=0000000000000000 bytes_per_launch=1\n"
                   f"kernel=admm_ul_u32_tc5 src={src} bytes_per_launch=333021184 read=1 write=2\n")
    assert bench.recorded_traffic("admm_ul_u32_tc5") == 333021184.0
    assert bench.recorded_traffic("admm_dl") is None
    assert bench.recorded_traffic("no_such_kernel") is None
    _append(tree / "paper_1702_04458_b300" / "csrc" / "dbp_tc32.cuh", "\n__device__ int changed;\n")
    assert bench.recorded_traffic("admm_ul_u32_tc5") is None
