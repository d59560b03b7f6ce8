"""Host logic of bench.py (no GPU): the kernel-source hash that ties the
committed ncu summary to the code ignores comments and layout but not code,
and the committed summary's traffic figure applies to the current source."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_code_only_ignores_comments_and_layout():
    a = "int f(int x) {\n  // one\n  return x + 1; /* two\n lines */\n}\n"
    b = "int f(int x) { return x + 1; }  // other comment"
    c = "int f(int x) { return x + 2; }"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)


def test_profile_summary_matches_the_current_kernel_source():
    """The committed headline summary was taken on the code as it stands, so
    the bench line reports its DRAM traffic (not null): about the 124.4 MB a
    3840x2160x3 uint8 launch must move (input read once, output written
    once)."""
    t = bench.profiled_traffic()
    assert t is not None and 1.15e8 < t < 1.40e8


def test_cpu_model_and_oracle_sample():
    import numpy as np
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()
    A = np.arange(3 * 40 * 7, dtype=float).reshape(3, 40, 7)
    win, r0 = bench.oracle_sample(A, 10)
    assert win.shape == (3, 19, 7)
    assert np.array_equal(win[:, 4], A[:, r0])


def test_kernel_sha_changes_with_the_code(tmp_path, monkeypatch):
    srcs = []
    for i, rel in enumerate(bench.KERNEL_SOURCES):
        p = tmp_path / f"k{i}.cuh"
        p.write_text(open(os.path.join(ROOT, rel), encoding="utf-8").read())
        srcs.append(str(p))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", srcs)
    monkeypatch.setattr(bench, "ROOT", "/")
    h0 = bench.kernel_sha()
    with open(srcs[0], "a", encoding="utf-8") as fh:
        fh.write("\n// a comment only\n")
    assert bench.kernel_sha() == h0
    with open(srcs[0], "a", encoding="utf-8") as fh:
        fh.write("\nstatic int extra_symbol;\n")
    assert bench.kernel_sha() != h0
