"""Host-side tooling of the benchmark and the profiles, on CPU: the ncu
launch-list summary, the clock sampler's parsing and the digit-pair count of
the emulated contractions, and that the tcgen05.mma rate probe builds."""
import io
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1704_07458_gb300 import profiling  # noqa: E402
import bench  # noqa: E402


def test_summarize_launches(tmp_path):
    f = tmp_path / "launches.csv"
    f.write_text(
        '==PROF== some banner line\n'
        '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream",'
        '"Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit",'
        '"Metric Value"\n'
        '"0","1","python","h","void lob::(anonymous namespace)::spmm_kernel<4>(long, int)",'
        '"1","7","(256,1,1)","(64,1,1)","0","10.3","Command line profiler metrics",'
        '"gpu__time_duration.sum","usecond","10.5"\n'
        '"1","1","python","h","void lob::(anonymous namespace)::spmm_kernel<4>(long, int)",'
        '"1","7","(256,1,1)","(64,1,1)","0","10.3","Command line profiler metrics",'
        '"gpu__time_duration.sum","nsecond","1,500"\n'
        '"2","1","python","h","lob::update_tc_kernel<6>(int)",'
        '"1","7","(256,1,1)","(64,1,1)","0","10.3","Command line profiler metrics",'
        '"gpu__time_duration.sum","msecond","0.088"\n')
    out = io.StringIO()
    tot, cnt = profiling.summarize_launches(str(f), out)
    assert cnt == {"lob::spmm_kernel": 2, "lob::update_tc_kernel": 1}
    assert tot["lob::spmm_kernel"] == pytest.approx(12.0)
    assert tot["lob::update_tc_kernel"] == pytest.approx(88.0)
    text = out.getvalue()
    assert "88.0%" in text and "12.0%" in text


def test_digit_pairs():
    # pairs (s, t) with s, t >= 1 and s + t <= S + 1: S (S + 1) / 2
    for S in range(1, 8):
        assert profiling.pairs(S) == S * (S + 1) // 2
    assert profiling.pairs(0) == 0


def test_clock_sampler_parses_reasons(tmp_path):
    c = bench.ClockSampler(0)
    with open(c.file.name, "w") as fh:
        fh.write("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        fh.write("0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        fh.write("0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        fh.write("garbage line\n")

    class Done:
        def terminate(self):
            pass

        def wait(self):
            pass

    c.proc = Done()
    r = c.stop()
    assert r["sm_mhz"] == 2070 and r["sm_max_mhz"] == 2070 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]


def test_mma_rate_probe_compiles(tmp_path):
    """The standalone tcgen05.mma rate probe behind `profiling mma-rate`
    builds for sm_103a (it runs only on a GB300)."""
    import shutil
    import subprocess
    from paper_1704_07458_gb300 import build as b
    try:
        nvcc = b._nvcc()
    except RuntimeError:
        pytest.skip("nvcc not found")
    src = os.path.join(os.path.dirname(b.__file__), "csrc", "probes", "tcgen05_mma_rate.cu")
    out = str(tmp_path / "tcgen05_mma_rate")
    subprocess.run([nvcc, *b.ARCH, "-O3", "-o", out, src], check=True)
    assert os.path.exists(out)
