"""Host-side logic of the serving loop (CPU only): the synthetic request stream, the per-session
camera paths, the admission footprint and the latency statistics."""
import math

import numpy as np

from paper_0811_2055_gb300 import serve


def test_poisson_requests_are_deterministic_and_have_the_offered_rate():
    res_choices = [(1280, 720), (1920, 1080), (3840, 2160)]
    r1, q1 = serve.poisson_requests(64, 30.0, 10.0, 16, res_choices, seed=0)
    r2, q2 = serve.poisson_requests(64, 30.0, 10.0, 16, res_choices, seed=0)
    assert r1 == r2 and [(q.session, q.arrival, q.timestep) for q in q1] == [(q.session, q.arrival, q.timestep) for q in q2]
    expected = 64 * 30.0 * 10.0
    assert abs(len(q1) - expected) < 5 * math.sqrt(expected)
    arr = [q.arrival for q in q1]
    assert arr == sorted(arr) and 0.0 <= arr[0] and arr[-1] < 10.0
    assert set(r1) <= set(res_choices) and len(set(r1)) == 3
    # each session starts at some timestep and advances one every 2 s
    for s in range(64):
        qs = [q for q in q1 if q.session == s]
        t0 = (qs[0].timestep - int(qs[0].arrival // 2.0)) % 16
        assert all(q.timestep == (t0 + int(q.arrival // 2.0)) % 16 for q in qs)
        assert all(q.camera["width"] == r1[s][0] and q.camera["height"] == r1[s][1] for q in qs)


def test_session_cameras_are_smooth_orthonormal_and_look_at_the_centre():
    for sid in range(5):
        a = serve.session_camera(sid, 1.0, 320, 200)
        b = serve.session_camera(sid, 1.0 + 1.0 / 30.0, 320, 200)
        assert np.linalg.norm(np.subtract(a["eye"], b["eye"])) < 0.05
        R = np.array([a["right"], a["up"], a["fwd"]])
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-12)
        to_c = np.subtract((0.5, 0.5, 0.5), a["eye"])
        assert np.allclose(np.asarray(a["fwd"]), to_c / np.linalg.norm(to_c), atol=1e-12)


def test_admission_footprint_and_latency_statistics():
    # a session holds `slots` frame buffers: a uint64 accumulator and an 8-bit image per slot
    assert serve.ServingLoop.session_bytes(1920, 1080, 2) == 2 * 1920 * 1080 * 9
    done = []
    for i in range(100):
        q = serve.Request(session=i % 3, arrival=0.01 * i, timestep=0, camera={})
        q.ready = q.arrival + 0.001 * (i + 1)
        done.append(q)
    st = serve.latency_stats(done, 1.0)
    lat = np.arange(1, 101) * 1.0
    assert st["completed"] == 100
    assert abs(st["p50_ms"] - np.percentile(lat, 50)) < 1e-9 and abs(st["p99_ms"] - np.percentile(lat, 99)) < 1e-9
    assert abs(st["frames_per_s"] - 100 / 1.09) < 1e-9
    assert serve.latency_stats([], 1.0) == {"completed": 0}
