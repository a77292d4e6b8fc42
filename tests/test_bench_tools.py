"""bench.py's host-side tools (CPU): the ncu-CSV to stage-traffic summary, and the
stage-source digest that keys it."""
import json
import os

import bench


def test_traffic_summary_sums_kernels_per_stage(tmp_path):
    """Two stages of the four stage kernels: per-kernel sums over the launches, per-stage
    bytes = total / stages, names stripped of their argument lists and return types."""
    header = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
              '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n')
    rows = []
    kernels = ["unnamed>::interior_kernel(Geo, StageArgs)", "void unnamed>::shell_kernel<0>(Geo, StageArgs)",
               "void unnamed>::pml_face_kernel<0>(Geo, StageArgs)",
               "void unnamed>::pml_kernel<0, 2, 3>(Geo, StageArgs, unnamed>::Region)"]
    lid = 0
    for stage in range(2):
        for k in kernels:
            for m, v in (("dram__bytes_read.sum", 100 + stage), ("dram__bytes_write.sum", 10),
                         ("gpu__time_duration.sum", 1000)):
                rows.append(f'"{lid}","1","python","h","{k}","1","1","(32, 8, 1)","(1, 1, 1)","0","10.3",'
                            f'"Command line profiler metrics","{m}","byte","{v}"\n')
            lid += 1
    path = tmp_path / "t.csv"
    path.write_text("==PROF== noise\n" + header + "".join(rows) + "==PROF== Disconnected\n")
    rec = bench.traffic_summary(str(path), "layered_96x96x48")
    assert rec["kernel_launches_captured"] == 8 and rec["stages_captured"] == 2
    assert sorted(rec["per_kernel"]) == ["unnamed>::interior_kernel", "unnamed>::pml_face_kernel<0>",
                                         "unnamed>::pml_kernel<0, 2, 3>", "unnamed>::shell_kernel<0>"]
    assert rec["per_kernel"]["unnamed>::interior_kernel"]["dram__bytes_read.sum"] == 201
    assert rec["dram_read_bytes_per_stage"] == 201 * 4 / 2 and rec["dram_write_bytes_per_stage"] == 40
    assert rec["dram_bytes_per_stage"] == rec["dram_read_bytes_per_stage"] + rec["dram_write_bytes_per_stage"]
    assert rec["csrc_sha256"] == bench.kernel_sources_sha256()


def test_committed_traffic_summary_matches_the_sources():
    """The committed summary is keyed to the stage-kernel sources: while they match, the
    bench reports its traffic; once they change, the bench reports null, and this test
    says so (a skip, since only a GPU capture can refresh it)."""
    import pytest

    path = os.path.join(bench.ROOT, "profiles", "stage_traffic_layered_96x96x48.json")
    with open(path) as f:
        rec = json.load(f)
    if rec["csrc_sha256"] != bench.kernel_sources_sha256():
        assert bench.measured_traffic("layered_96x96x48", 1) is None
        pytest.skip("stage-kernel sources changed since the traffic capture: rerun bench.TRAFFIC_COMMAND on a "
                    "GPU and python bench.py --traffic-json on its CSV")
    assert bench.measured_traffic("layered_96x96x48", 1) == rec["dram_bytes_per_stage"]
