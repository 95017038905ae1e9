"""The defaults follow the values the paper prints (Sec. IV-A, fixture
tests/golden/paper_hyperparameters.json): the global loop retrieval's two
thresholds, the keyframe buffer of N frames per submap, and the 518-pixel
long side of the synthetic frames and of the benchmark's chain."""
import inspect
import json
import os

import bench
from paper_2510_02080_b300 import ec3r, synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_hyperparameters.json")


def paper():
    with open(GOLDEN) as f:
        return {k: v["value"] for k, v in json.load(f).items()}


def test_loop_retrieval_thresholds():
    p = paper()
    sig = inspect.signature(ec3r.Context.loop_candidates)
    assert sig.parameters["tau_global"].default == p["tau_global"]
    assert sig.parameters["tau_local"].default == p["tau_local"]


def test_submap_frames_and_image_size():
    p = paper()
    for fn in (synth.make_chain, synth.make_depth_chain):
        sig = inspect.signature(fn)
        assert sig.parameters["F"].default == p["keyframe_buffer_N"]
        assert sig.parameters["W"].default == p["image_long_side"]
    assert inspect.signature(synth.make_loop_batch).parameters["max_frames"].default == \
        p["keyframe_buffer_N"]
    assert bench.F_FRAMES == p["keyframe_buffer_N"]
    assert max(bench.H, bench.W) == p["image_long_side"]
