"""The GPU tests predict which kernel serves a pass (and so how many launches
an application takes) from the plan's fixed kernel-choice rules.  Those rules
live in the CUDA sources as constants; this CPU test keeps the tests' copies
of them equal to the sources, so that a change of a rule cannot leave the
launch-count and kernel-selection tests checking a stale rule."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1404_5756_gb300", "csrc")


def constant(path, name):
    text = open(os.path.join(CSRC, path)).read()
    m = re.search(r"constexpr\s+(?:int|int64_t)\s+" + name + r"\s*=\s*(\d+)\s*;", text)
    assert m, f"{name} not found in {path}"
    return int(m.group(1))


def source_of(name):
    return open(os.path.join(ROOT, "tests", name + ".py")).read()


def literal(src, name):
    m = re.search(r"^" + name + r"\s*=\s*(\d+)", src, flags=re.M)
    assert m, name
    return int(m.group(1))


def test_streaming_kernel_rules_match_the_sources():
    max_ends = constant("rf_stream.cuh", "kStreamMaxEnds")
    min_work = constant("rf_plan.cu", "kStreamMinWork")
    batch = source_of("test_gpu_batch")
    stream = source_of("test_gpu_stream")
    assert literal(batch, "STREAM_MAX_ENDS") == max_ends
    assert literal(batch, "STREAM_MIN_WORK") == min_work
    assert literal(stream, "MAX_ENDS") == max_ends
    assert literal(stream, "MIN_WORK") == min_work


def test_register_kernel_line_limit_matches_the_batch_test():
    """The batch test sends lines of at most 1024 points to the register
    kernel; the planner's limit is the longest built shape, P C = 1024."""
    text = open(os.path.join(CSRC, "rf_reg_launch.h")).read()
    table = text.split("kRegShapes[]")[1].split(";")[0]
    shapes = [(int(c), int(p)) for c, p in re.findall(r"\{(\d+),\s*(\d+)\}", table)]
    assert max(c * p for c, p in shapes) == 1024
    plan = open(os.path.join(CSRC, "rf_plan.cu")).read()
    assert re.search(r"q\.n > 1024\) return RegShape\{0, 0\}", plan)
    assert "m <= 1024" in source_of("test_gpu_batch")
