"""chem_integrate_cells_noalloc through the C ABI: two calls in a row give the result of
chem_integrate_cells on the same inputs, leave the device's free memory unchanged, and
reject a mechanism whose workspace exceeds the static scratch.  Collected last; also passes
alone in a fresh process."""
import numpy as np
import pytest
import torch

from paper_2008_08483_gb300 import build as B
from paper_2008_08483_gb300 import chem, synth

pytestmark = pytest.mark.gpu


def _call(h, T, P, Y, status, t_end):
    """chem_integrate_cells_noalloc on the current stream, all arrays pre-allocated."""
    L = chem.lib()
    return L.chem_integrate_cells_noalloc(h.handle, T.shape[0], T.data_ptr(), P.data_ptr(),
                                          Y.data_ptr(), Y.stride(0), t_end, 1e-6, 1e-12, None,
                                          status.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream)


def test_noalloc_matches_integrate_cells():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.build()
    dev = torch.device("cuda:0")
    m = synth.make_mechanism("gri_53_325", seed=1)
    h = chem.Mechanism(m)
    T, P, Y, _ = synth.make_ignition_states(m, 300, seed=77)
    args = lambda: [torch.as_tensor(a, dtype=torch.float64, device=dev).clone() for a in (T, P, Y)]
    Tr, Pr, Yr = args()
    ref = chem.integrate(h, Tr, Pr, Yr, 2e-6, stats=False)
    assert not ref["failed"]
    status = torch.full((300,), -1, dtype=torch.int32, device=dev)
    for it in range(2):                              # two calls in a row share the scratch
        Ta, Pa, Ya = args()
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        assert _call(h, Ta, Pa, Ya, status, 2e-6) == 0, chem.lib().chem_last_error()
        torch.cuda.synchronize()
        if it == 1:
            # after the first call's set-up (which may load the module holding the static
            # array), a call leaves the device's free memory unchanged
            assert torch.cuda.mem_get_info()[0] == free_before
        assert int((status != 0).sum()) == 0
        assert np.allclose(Ta.cpu().numpy(), Tr.cpu().numpy(), rtol=1e-12, atol=0)
        assert np.allclose(Ya.cpu().numpy(), Yr.cpu().numpy(), rtol=1e-12, atol=1e-300)
        del Ta, Pa, Ya
    h.close()


@pytest.mark.parametrize("n", [1, 64])
def test_noalloc_rejects_workspace_beyond_scratch(n):
    """A mechanism whose reactor matrices exceed shared memory is refused for any cell
    count, a single cell included: the limit belongs to the mechanism."""
    B.build()
    dev = torch.device("cuda:0")
    m = synth.make_mechanism("heavy_160_1000", seed=1)   # reactor matrices exceed shared memory
    h = chem.Mechanism(m)
    T, P, Y, _ = synth.make_ignition_states(m, n, seed=3)
    Tt, Pt, Yt = (torch.as_tensor(a, dtype=torch.float64, device=dev) for a in (T, P, Y))
    status = torch.zeros((n,), dtype=torch.int32, device=dev)
    assert _call(h, Tt, Pt, Yt, status, 1e-9) == 2                # CHEM_ENOMEM
    assert b"static scratch" in chem.lib().chem_last_error()
    assert np.array_equal(Tt.cpu().numpy(), T)     # nothing ran
    h.close()
