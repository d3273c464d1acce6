"""Serving admission timeout: with one slot, the first request is admitted
and served (its result equal, bit for bit, to the model on its input alone);
the two behind it wait past the timeout, are dropped at the next step, which
counts them as finished, and report FHEON_ERR_TIMEOUT; a bad timeout is
refused."""
import time

import pytest

import gpu_common
from oracle import ckks
from oracle import fheon as OF
from paper_2510_03996_gb300 import synth

pytestmark = pytest.mark.gpu

GRID, BLOCK = 8, 64


def test_requests_waiting_past_the_timeout_are_dropped():
    pr = gpu_common.Pair("relu_n12")
    g, F, D = pr.g, pr.F, pr.P["scale"]
    K = synth.conv_kernel(96, 0, (2, 1, 3, 3), std=0.3)
    conv = g.conv_prepare((1, 6, 6, GRID, 1, BLOCK), K, 1, pr.L, D, bias=[0.1, -0.1])
    pr.add_keys(g.layer_rotation_steps(conv))
    model = g.model([conv])
    cts = []
    for i in range(3):
        v = OF.pack_map(synth.image(96, 10 + i, (1, 6, 6)), pr.N // 2, GRID, 1, BLOCK)
        cts.append(pr.encrypt_both(ckks.encode(v, pr.N, D), nonce=9600 + i)[0])
    alone = g.ct_download(g.model_run(model, cts[0]))

    srv = g.server(max_active=1)
    with pytest.raises(F.FheonError) as e:
        srv.set_admit_timeout(-1.0)
    assert e.value.code == -1
    srv.set_admit_timeout(0.5)
    ids = [srv.submit(model, ct) for ct in cts]
    assert srv.step() == 1                     # request 0: admitted, one layer, done
    assert srv.stats()["waiting"] == 2
    time.sleep(0.6)
    assert srv.step() == 2                     # the other two: dropped
    assert srv.stats()["waiting"] == 0 and srv.stats()["active"] == 0
    assert gpu_common.mismatch(g.ct_download(srv.result(ids[0])), alone) == 0
    for rid in ids[1:]:
        with pytest.raises(F.FheonError) as e:
            srv.result(rid)
        assert e.value.code == -6 and "admission timeout" in str(e.value)
        with pytest.raises(F.FheonError):
            srv.result(rid)                    # forgotten after the report
    srv.close()
