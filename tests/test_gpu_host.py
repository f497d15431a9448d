"""chem_source_term_host (host arrays, chunked copy / kernel pipeline) against
chem_source_term on device arrays: identical results for every precision, contiguous and
padded output rows, ragged last chunk, chunk larger than the batch; argument errors."""
import numpy as np
import pytest
import torch

from paper_2008_08483_gb300 import build as B
from paper_2008_08483_gb300 import chem, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.build()
    m = synth.make_mechanism("gri_53_325", seed=1)
    h = chem.Mechanism(m)
    T, P, Y = synth.make_states(m, 5000, seed=8)
    return m, h, T, P, Y


@pytest.mark.parametrize("prec", [chem.FP64, chem.FP32, chem.SPLIT_BF16])
@pytest.mark.parametrize("chunk,ldO", [(1024, 53), (777, 53), (1024, 60), (9000, 53)])
def test_host_pipeline_matches_device_call(setup, prec, chunk, ldO):
    m, h, T, P, Y = setup
    dev = torch.device("cuda:0")
    dt = torch.float64 if prec == chem.FP64 else torch.float32
    n, ns = T.shape[0], m.n_species
    ref = chem.source_term(h, *(torch.as_tensor(a, dtype=dt, device=dev) for a in (T, P, Y)),
                           prec).cpu()
    hT, hP, hY = (torch.as_tensor(a, dtype=dt).pin_memory() for a in (T, P, Y))
    hO = torch.full((n, ldO), -7.0, dtype=dt).pin_memory()
    wsb = chem.host_workspace_bytes(h, min(chunk, n), ns, prec)
    work = torch.empty(wsb, dtype=torch.uint8, device=dev)
    chem.source_term_host(h, hT, hP, hY, hO, prec, work, chunk)
    torch.cuda.synchronize()
    assert torch.equal(hO[:, :ns], ref)
    if ldO > ns:
        assert torch.all(hO[:, ns:] == -7.0)             # padding columns untouched


def test_host_pipeline_errors(setup):
    m, h, T, P, Y = setup
    dev = torch.device("cuda:0")
    hT, hP, hY = (torch.as_tensor(a[:100], dtype=torch.float32).pin_memory() for a in (T, P, Y))
    hO = torch.empty((100, 53), dtype=torch.float32).pin_memory()
    wsb = chem.host_workspace_bytes(h, 64, 53, chem.FP32)
    small = torch.empty(wsb - 256, dtype=torch.uint8, device=dev)
    with pytest.raises(chem.ChemError) as e:
        chem.source_term_host(h, hT, hP, hY, hO, chem.FP32, small, 64)
    assert e.value.status == 1
    big = torch.empty(wsb + 512, dtype=torch.uint8, device=dev)
    L = chem.lib()
    rc = L.chem_source_term_host(h.handle, 100, hT.data_ptr(), hP.data_ptr(), hY.data_ptr(), 53,
                                 hO.data_ptr(), 53, chem.FP32, 64, big.data_ptr() + 16,
                                 wsb, None)
    assert rc == 1                                         # workspace not 256-byte aligned
    rc = L.chem_source_term_host(h.handle, 100, hT.data_ptr(), hP.data_ptr(), hY.data_ptr(), 53,
                                 hO.data_ptr(), 53, chem.FP32, 0, big.data_ptr(), wsb, None)
    assert rc == 1                                         # chunk_cells < 1
