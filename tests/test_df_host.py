"""Host check of the mixed path's double-float toolkit (qp_df.h): integer
split/merge of FP64 values, error-free transformations, double-float
arithmetic and chi_e's cancellation, against long-double arithmetic."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_double_float_toolkit(tmp_path):
    exe = tmp_path / "df_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I",
                    os.path.join(ROOT, "paper_1311_1107_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "df_check.cpp"), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    results = {line.split()[0]: int(line.split()[1]) for line in out.splitlines()}
    assert set(results) == {"split", "hi_d", "roundtrip", "add_fd", "merge", "f_to_d", "eft",
                            "arith", "chi_cancellation"}
    assert all(v == 0 for v in results.values()), out
