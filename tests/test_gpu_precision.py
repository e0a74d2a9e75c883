"""16-bit offset storage (FP16 / BF16 flow populations; adjoint and
temperature populations stay FP32; FP32 arithmetic): error against the FP64
oracle per field after fixed steps."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2501_02161_gb300 import inputs as I
from test_gpu_parity import rel, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

# stated bounds (rel-L2 vs the FP64 oracle after the fixed steps below)
BOUND = {"fp16": {"rho": 1e-3, "u": 5e-3, "T": 1e-2, "fs": 5e-3, "sens": 1e-2},
         "bf16": {"rho": 1e-2, "u": 5e-2, "T": 5e-2, "fs": 1e-2, "sens": 5e-2}}


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_02161_gb300 import build as B
    B.build()
    O.build()


RESULTS = {}


@pytest.mark.parametrize("storage", ["fp16", "bf16", "fp32"])
@pytest.mark.parametrize("lat", [I.pipe_bend_3d(n=24, width=6, re=20.0, seed=2),
                                 I.heat_sink(nx=32, ny=16, nz=12, re=20.0, q_flux=2e-3, seed=4)],
                         ids=lambda l: l.name)
def test_sixteen_bit_error_vs_oracle(lat, storage):
    g = run_gpu(lat, storage, 600, 400, K=200)
    o = run_oracle(lat, 600, 400)
    errs = {k: float(rel(g[k], o[k])) for k in ("rho", "u", "sens", "fs") + (("T",) if "T" in o else ())}
    RESULTS[f"{lat.name}/{storage}"] = errs
    out = os.environ.get("LBM_TEST_RECORDS")  # optional folder for the measured values
    if out and os.path.isdir(out):
        json.dump(RESULTS, open(os.path.join(out, "precision_errors.json"), "w"), indent=1)
    if storage in BOUND:
        for k, v in errs.items():
            assert np.isfinite(v) and v <= BOUND[storage][k], errs
