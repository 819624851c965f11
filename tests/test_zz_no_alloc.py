"""ds_reconstruct_noalloc: the entry point for callers that cannot allocate
device memory (a host framework owning all device allocations, code that must
not trigger an allocation's implicit synchronisation, callers that cannot
create a context).  Called through the C ABI, twice in a row, its tracks must
equal those of ds_reconstruct on the same batch within the parity tolerances.
This file is collected last on purpose: it uses the library's static scratch."""
import numpy as np
import pytest

from paper_2503_13092_b300 import synth
from tests import parity

pytestmark = pytest.mark.gpu


def test_noalloc_matches_reconstruct():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_13092_b300 import build, ds
    build.build()
    cfg = synth.default_config()
    w = synth.nn_weights()
    b = synth.config_batch("c2", n_events=40)
    d = ds.Downstream(cfg, w)
    ref = d.run(b)
    assert ref["n_tracks"] > 1000
    dev = d.to_device(b)
    E, S = dev["n_events"], dev["n_seeds"]
    geom = ds.make_geometry(cfg)
    params = ds.make_params(cfg)
    for call in range(2):
        out = d.alloc_tracks(E, S)
        flags = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = ds.ds_reconstruct_noalloc(geom, params, w, dev, out, d_flags=flags)
        assert st == ds.DS_OK, ds.ds_status_string(st)
        torch.cuda.synchronize()
        if call == 1:
            # the defining property: the call itself takes no device memory
            # (the first call may load the library's module on the device)
            assert torch.cuda.mem_get_info()[0] == free0
        assert int(flags.item()) == 0
        got = ds.decode(out)
        assert got["n_tracks"] == ref["n_tracks"]
        assert np.array_equal(got["trk_off"], ref["trk_off"])
        t, r = got["tracks"], ref["tracks"]
        assert np.array_equal(t["seed"], r["seed"]) and np.array_equal(t["hit"], r["hit"])
        for k in ("x", "y", "tx", "ty", "qop"):
            assert np.all(parity._close(t[k].astype(float), r[k].astype(float), parity.RTOL_PAR, parity.ATOL_PAR)), k
        assert np.all(parity._close(t["chi2"].astype(float), r["chi2"].astype(float), parity.RTOL_CHI2,
                                    parity.ATOL_CHI2))
        assert np.max(np.abs(t["nn"] - r["nn"])) <= parity.ATOL_NN
    # sizes beyond the static scratch are refused before anything runs
    big = dict(dev)
    big["n_events"] = 257
    out = d.alloc_tracks(E, S)
    assert ds.ds_reconstruct_noalloc(geom, params, w, big, out) == ds.DS_ERR_CAPACITY
    # training mode (up to 40 candidates per seed) does not fit the static buffer
    assert ds.ds_reconstruct_noalloc(geom, ds.make_params(cfg, training=1), w, dev, out) == ds.DS_ERR_ARG
    d.close()
