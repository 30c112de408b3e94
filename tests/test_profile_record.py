"""The bench line's DRAM traffic comes from the committed ncu summary of the
step kernel, and only while the kernel sources it was captured from are
unchanged (a source hash in the summary). These CPU checks keep the summary and
the sources in step: a change to the step kernel needs a new capture."""
import bench


def test_headline_profile_matches_kernel_sources():
    t = bench.traffic_record("f32_c")
    assert t is not None, "profiles/step_kernel_bubble_1024x4096.md was captured from other kernel sources"
    # within a factor of two of the algorithmic 176 bytes a cell (the replayed
    # launch leaves part of its writes in L2)
    cells = 1024 * 4096
    assert 0.5 * 176 * cells < t < 2.0 * 176 * cells


def test_unknown_form_has_no_record():
    assert bench.traffic_record("no_such_form") is None
