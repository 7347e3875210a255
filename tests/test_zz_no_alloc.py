"""The allocation-free Gram entry point (copa_gram_noalloc) against copa_gram.

copa_gram_noalloc exists for callers that must not allocate device memory while it runs
(their memory is reserved by their own pool, or an allocation's device synchronisation
would stall their other work). It keeps its scratch in a fixed device array owned by the
library, so two calls in a row reuse the same memory: both must still match copa_gram.
This file is collected last so that a failure here does not hide the other tests."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc_matches(P, dtype, shapes):
    import torch
    h = P.Copa(0, "mixed" if dtype == torch.float32 else "fp64")
    s = torch.cuda.Stream()
    rng = np.random.default_rng(17)
    for rows, R in shapes:                       # consecutive calls share the scratch array
        A = torch.as_tensor(rng.standard_normal((rows, R)), dtype=dtype, device="cuda")
        G_ref = h.gram(A)
        G = torch.full((R, R), float("nan"), dtype=torch.float64, device="cuda")
        s.wait_stream(torch.cuda.current_stream())
        P.gram_noalloc(A, G, s)
        torch.cuda.current_stream().wait_stream(s)
        h.sync()
        torch.cuda.synchronize()
        ref = G_ref.cpu().numpy()
        got = G.cpu().numpy()
        tol = 1e-10 if dtype == torch.float64 else 1e-5
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref), (rows, R)


def test_gram_noalloc_matches_copa_gram_twice_fp64():
    import paper_1803_04572_gb300 as P
    import torch
    _noalloc_matches(P, torch.float64, [(70001, 40), (5003, 13)])


def test_gram_noalloc_matches_copa_gram_twice_fp32():
    import paper_1803_04572_gb300 as P
    import torch
    _noalloc_matches(P, torch.float32, [(120000, 40), (999, 90)])


def test_gram_noalloc_rejects_too_large_rank():
    import paper_1803_04572_gb300 as P
    import torch
    A = torch.zeros((10, 91), dtype=torch.float32, device="cuda")
    G = torch.zeros((91, 91), dtype=torch.float64, device="cuda")
    with pytest.raises(P.CopaError) as e:
        P.gram_noalloc(A, G, torch.cuda.Stream())
    assert e.value.code == P.ERR_UNSUPPORTED
