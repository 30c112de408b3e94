"""The bench line's DRAM traffic comes from the committed ncu summary of the
step kernel, and only while the kernel sources it was captured from are
unchanged (a source hash in the summary); after a change the bench reports
traffic as null until a new capture is committed. These CPU checks keep that
rule honest: a record whose hash matches must be a plausible per-launch byte
count, and one whose hash does not match must read as None."""
import hashlib
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUMMARY = os.path.join(ROOT, "profiles", "step_kernel_bubble_1024x4096.md")


def _sources_sha():
    h = hashlib.sha256()
    for name in ("lbm_device.cuh", "lbm_step_x2.cuh"):
        with open(os.path.join(ROOT, "paper_1902_08933_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def test_headline_profile_record_is_fresh_or_null():
    text = open(SUMMARY).read()
    m = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    assert m, "the summary names the source hash it was captured from"
    t = bench.traffic_record("f32_c")
    if m.group(1) == _sources_sha():
        # within a factor of two of the form's 176 bytes a cell (the replayed
        # launch leaves part of its writes in L2)
        cells = 1024 * 4096
        assert t is not None and 0.5 * 176 * cells < t < 2.0 * 176 * cells
    else:
        assert t is None


def test_unknown_form_has_no_record():
    assert bench.traffic_record("no_such_form") is None
