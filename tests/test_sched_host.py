"""CPU test of the serving loop's scheduling (paper_2206_06302_b300/csrc/sx_sched.h): the arena
allocator against a byte-level model and the step planner's three policies, through the C++
program tests/sched_host_test.cpp (no GPU, no CUDA)."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_arena_and_step_planner(tmp_path):
    exe = str(tmp_path / "sched_host_test")
    subprocess.run(["g++", "-std=c++17", "-O2", "-Wall", "-Wextra", "-Werror",
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2206_06302_b300", "csrc"),
                    os.path.join(ROOT, "tests", "sched_host_test.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)
