"""The tile autotuner on the GPU: it times every candidate, installs the fastest, caches it per
workload bucket, and the installed choice leaves results bit-identical."""
import json

import numpy as np
import pytest

from paper_2104_04582_gb300 import fewsum as F
from paper_2104_04582_gb300 import runtime as RT
from paper_2104_04582_gb300 import tune
from paper_2104_04582_gb300 import workloads as W
from tests.gpu_common import to_host

pytestmark = pytest.mark.gpu


def test_tune_installs_and_caches_a_choice(gpu_ctx, tmp_path):
    import torch
    w = W.config1()
    tr = RT.from_inputs(gpu_ctx, w)
    out = RT.alloc_out(w.n_samples, True)
    saved = gpu_ctx.get_tiles(F.FEW_MIXED)
    ref = to_host(RT.waveform_inputs(gpu_ctx, tr, w, F.FEW_MIXED))
    cache = str(tmp_path / "tiles.json")
    run = lambda: RT.waveform_inputs(gpu_ctx, tr, w, F.FEW_MIXED, out=out)
    K, N, slots = tr.info
    try:
        best, times = tune.tune(gpu_ctx.handle, run, F.FEW_MIXED, slots, w.n_samples, repeats=2,
                                cache_path=cache)
        assert len(times) == len(tune.CANDIDATES[F.FEW_MIXED])
        assert gpu_ctx.get_tiles(F.FEW_MIXED) == tuple(best)
        data = json.load(open(cache))
        key = tune.bucket(F.FEW_MIXED, slots, w.n_samples)
        assert (data[key]["R"], data[key]["threads"], data[key]["stage_slots"]) == tuple(best)
        run()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(to_host(out), ref)
        gpu_ctx.set_tiles(F.FEW_MIXED, 2, 128, 16)
        assert tune.apply_cached(gpu_ctx.handle, F.FEW_MIXED, slots, w.n_samples, cache) == best
        assert gpu_ctx.get_tiles(F.FEW_MIXED) == tuple(best)
        gpu_ctx.set_tiles(F.FEW_MIXED, 2, 128, 16)
        assert tune.ensure(gpu_ctx.handle, run, F.FEW_MIXED, slots, w.n_samples, cache) == (best, False)
    finally:
        gpu_ctx.set_tiles(F.FEW_MIXED, *saved)
        tr.release()
