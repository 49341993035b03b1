"""Storage precision vs arithmetic precision on the small STAI workload (GPU).

The same physical RF stored as float32, float16 or int16: the GPU result must
match the FP64 oracle run on the *stored* values within the FP32 arithmetic
bar (rel-L2 <= 1e-4) for every storage type, while the storage error itself
(oracle on stored vs oracle on the unrounded synthesis) is reported, not
bounded by that bar.  tests/precision_report.py tabulates the same split for
the full workloads.
"""
import numpy as np
import pytest

import oracle
from helpers import THREADS, TOL_BF_REL_L2, das_gpu, rel_l2
from synth import configs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f32", "f16", "i16"])
def test_arithmetic_error_independent_of_storage(dtype):
    base = configs.stai_small()
    case = configs._with_rf(base, base.meta["rf_f64"], dtype)
    got = das_gpu(case).cpu().numpy()[0]
    on_stored = oracle.das(case, threads=THREADS)
    pr, gr = oracle.probe_grid(case)
    on_true = oracle.das_stai(case.meta["rf_f64"][0], pr, gr, threads=THREADS)
    assert rel_l2(got, on_stored) <= TOL_BF_REL_L2
    storage = rel_l2(on_stored, on_true)
    bound = {"f32": 1e-7, "f16": 2e-3, "i16": 2e-3}[dtype]
    assert storage <= bound, (dtype, storage)
