"""CPU checks of the C-ABI library: exports, host-only entry points, and the
sorting-network tables compiled by the host compiler. No GPU is touched."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vqsort.h")
CSRC = os.path.join(ROOT, "paper_2205_05982_gb300", "csrc")


@pytest.fixture(scope="module")
def lib():
    from paper_2205_05982_gb300 import _build
    import paper_2205_05982_gb300 as vq
    _build.build()
    return vq.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(vqsort_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (vqsort_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_status_strings_and_options(lib):
    import paper_2205_05982_gb300 as vq
    assert vq.status_string(0) == "ok"
    assert "timeout" in vq.status_string(5) or "wait" in vq.status_string(5)
    old = vq.get_option("depth_limit")
    vq.set_option("depth_limit", 3)
    assert vq.get_option("depth_limit") == 3
    vq.set_option("depth_limit", old)
    assert vq.get_option("host_direct") == 0      # copy engines bring host results back by default
    vq.set_option("host_direct", 1)
    assert vq.get_option("host_direct") == 1
    vq.set_option("host_direct", 0)
    with pytest.raises(vq.VqError):
        vq.set_option("leaf_cutoff", 1000)      # not a power of two
    with pytest.raises(vq.VqError):
        vq.set_option("depth_limit", -5)


def test_argument_checks_before_any_device_call(lib):
    """Bad arguments are rejected on the host, before any CUDA call."""
    assert lib.vqsort_sort(99, None, 10, 1, None) == 1                       # bad dtype
    assert lib.vqsort_sort(6, None, 10, 1, None) == 1                        # null with n > 0
    assert lib.vqsort_sort(6, ctypes.c_void_p(0x1004), 10, 1, None) == 1     # misaligned u64
    assert lib.vqsort_sort(8, ctypes.c_void_p(0x1008), 10, 1, None) == 1     # u128 needs 16 B
    assert lib.vqsort_sort(6, ctypes.c_void_p(0x1000), 1, 1, None) == 0      # n <= 1: no-op
    assert lib.vqsort_sort(6, None, 0, 1, None) == 0
    assert lib.vqsort_choose_pivot(6, ctypes.c_void_p(0x1000), 100, 1, 1, ctypes.c_void_p(8), None) == 1


def test_workspace_bytes_grows_with_n(lib):
    import paper_2205_05982_gb300 as vq
    a = vq.workspace_bytes("u64", 10**6)
    b = vq.workspace_bytes("u64", 10**8)
    assert a >= 8 * 10**6 and b >= 8 * 10**8 and b > a
    assert vq.workspace_bytes("u64", 10**6, 1000) > a


def test_workspace_bytes_monotone_across_the_size_rules(lib):
    """A workspace sized for N keys covers every sort of n <= N keys: the
    default leaf cutoff and tile window change with n (16384 / 8192 / 4096
    keys; 16 KiB windows for short arrays), so the size must still grow with
    n across their bounds, for one array and for segmented batches."""
    import paper_2205_05982_gb300 as vq
    points = set()
    for b in (1 << 21, 1 << 22, 1 << 25, 1 << 26):
        points.update((b - 1, b, b + 1))
    points.update((2, 1000, 4096, 16384, 65536, 10**6, 10**7, 10**8, 3 * 10**8))
    points = sorted(points)
    for dt in ("i16", "u32", "f32", "u64", "f64", "u128", "kv64"):
        for segs in (1, 64):
            sizes = [vq.workspace_bytes(dt, n, segs) for n in points]
            assert all(x <= y for x, y in zip(sizes, sizes[1:])), (dt, segs, list(zip(points, sizes)))


def _golden_pairs(name):
    rows = []
    for line in open(os.path.join(ROOT, "tests", "golden", name)):
        line = line.strip()
        if line and not line.startswith("#"):
            v = [int(x) for x in line.split()]
            rows.append([(v[i], v[i + 1]) for i in range(0, len(v), 2)])
    return rows


@pytest.mark.parametrize("keys_per_thread", [1, 2, 4])
def test_merge_schedule_matches_paper_example(lib, keys_per_thread):
    """The networks' merge of two sorted runs of 4 keys runs exactly the
    modules printed in Sec. 3, whatever the keys-per-thread split."""
    import paper_2205_05982_gb300 as vq
    want = [sorted((a - 1, b - 1) for a, b in step) for step in _golden_pairs("bitonic_merge_2x4.txt")]
    got = [sorted(step) for step in vq.merge_schedule(4, keys_per_thread)]
    assert got == want


def test_networks_zero_one_principle(tmp_path):
    """Compiles networks.h with the host compiler and checks every column
    network and every merge schedule on all 0/1 inputs."""
    exe = tmp_path / "net_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "net_check.cpp"),
                    "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout
    assert "sizes 1 5 19 60" in r.stdout and r.stdout.strip().endswith("ok")


def test_stats_struct_matches_header():
    """The binding's vq_stats fields are the header's, in order."""
    from paper_2205_05982_gb300 import Stats
    with open(os.path.join(ROOT, "include", "vqsort.h")) as f:
        text = f.read()
    body = text[text.index("typedef struct vq_stats {"):text.index("} vq_stats;")]
    names = re.findall(r"uint64_t\s+(\w+);", body)
    assert names == [f for f, _ in Stats._fields_]
