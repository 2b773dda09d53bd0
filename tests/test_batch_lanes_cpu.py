"""CPU checks of the batched runner's split of streams over CUDA-stream lanes
(BatchRunner.lane_sets): every stream lands in exactly one lane, lanes keep
stream order inside, no lane is empty, and the pixel loads are balanced by
the largest-first rule."""
from types import SimpleNamespace

import pytest

from paper_1702_05156_gb300.batch import BatchRunner

SIZES = [(320, 240)] * 16 + [(640, 480)] * 16 + [(1280, 720)] * 16 + [(1920, 1080)] * 16


def _sets(specs, lanes):
    return BatchRunner.lane_sets(SimpleNamespace(specs=specs), lanes)


@pytest.mark.parametrize("lanes", [1, 2, 3, 4, 8])
def test_every_stream_once_and_balanced(lanes):
    specs = [(w, h, 4 if i % 3 else 8) for i, (w, h) in enumerate(SIZES)]
    sets = _sets(specs, lanes)
    assert len(sets) == lanes
    flat = sorted(i for s in sets for i in s)
    assert flat == list(range(len(specs)))
    for s in sets:
        assert s == sorted(s) and s
    loads = [sum(specs[i][0] * specs[i][1] for i in s) for s in sets]
    # largest first onto the lightest lane: no lane exceeds the mean by more
    # than the largest stream
    largest = max(w * h for (w, h, _) in specs)
    assert max(loads) - sum(loads) / lanes <= largest


def test_more_lanes_than_streams():
    specs = [(320, 240, 4), (640, 480, 8)]
    sets = _sets(specs, 8)
    assert sorted(i for s in sets for i in s) == [0, 1]
    assert all(s for s in sets) and len(sets) == 2


def test_equal_streams_split_evenly():
    specs = [(1920, 1080, 4)] * 8
    assert [len(s) for s in _sets(specs, 4)] == [2, 2, 2, 2]


def test_launch_shape_fills_the_abi_options():
    """LaunchShape.opts() fills dmsgm_batch_opts field by field (reserved 0,
    ctas, use_pdl, item_warps), in the header's order."""
    import ctypes

    from paper_1702_05156_gb300 import _lib
    from paper_1702_05156_gb300.batch import LaunchShape
    o = LaunchShape(1 << 30, True, 2, 8).opts()
    assert (o.reserved, o.ctas, o.use_pdl, o.item_warps) == (0, 1 << 30, 1, 8)
    o = LaunchShape().opts()
    assert (o.reserved, o.ctas, o.use_pdl, o.item_warps) == (0, 0, 1, 0)
    # the binding's fields are the header's, in its order
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "include", "dmsgm.h")).read()
    end = hdr.index("} dmsgm_batch_opts;")
    body = hdr[hdr.rindex("typedef struct {", 0, end) + len("typedef struct {"):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"int\s+(\w+)\s*;", body)
    assert [f for f, _ in _lib.dmsgm_batch_opts._fields_] == names == [
        "reserved", "ctas", "use_pdl", "item_warps"]
    assert ctypes.sizeof(_lib.dmsgm_batch_opts) == 4 * len(names)
