"""Serving loop on the GPU: every result of a mixed stream (several workers, overlapping on
the device, resident handles reused across requests of one shape) is bitwise equal to the
same request solved alone on a fresh handle."""
import numpy as np
import pytest

from tests.helpers import build_and_load, have_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not have_gpu(), reason="needs a CUDA GPU")]


def test_mixed_stream_results_equal_solo_results():
    build_and_load()
    from paper_2602_13841_gb300.serving import Request, Server, report
    reqs = [Request(0, 2, 16, 1, 1, 150.0, "TG2D"), Request(1, 2, 8, 2, 2, 900.0, "MMS2D"),
            Request(2, 2, 16, 1, 1, 1200.0, "MMS2D"), Request(3, 3, 4, 1, 1, 400.0, "TG3D"),
            Request(4, 2, 12, 3, 0, 300.0, "TG2D"), Request(5, 2, 16, 1, 1, 700.0, "TG2D"),
            # 3D shapes whose kernels share template instances with different shared-memory needs
            Request(6, 3, 4, 1, 2, 500.0, "MMS3D"), Request(7, 3, 4, 1, 0, 300.0, "TG3D"),
            Request(8, 3, 4, 2, 1, 800.0, "TG3D")]
    mix = Server(workers=3, keep_solutions=True)
    res = mix.run(reqs, realtime=False)
    mix.close()
    assert all(r.status == 0 for r in res), [(r.status, r.error) for r in res]
    rep = report(res)
    assert rep["completed"] == len(reqs) and rep["p99_s"] >= rep["p50_s"]
    for q, r in zip(reqs, res):
        solo = Server(workers=1, keep_solutions=True)
        s = solo.run([q], realtime=False)[0]
        solo.close()
        assert s.status == 0
        assert np.array_equal(s.solution, r.solution), q
