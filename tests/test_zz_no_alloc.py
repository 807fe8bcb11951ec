"""GPU check of idos_eval_idos_noalloc, the entry point for callers that cannot
allocate device memory (a framework that owns every device allocation through
its own pool, or a latency-critical loop that must not pay cudaMalloc's
implicit synchronisation).  Its scratch is a static device array; this test
calls it through the C ABI twice in a row and compares both results with the
ordinary allocating entry point idos_eval_idos.  Collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pkg = pytest.importorskip("paper_1611_09784_gb300")
from paper_1611_09784_gb300 import binding  # noqa: E402

from gpu_common import EIG_TOL, IDOS_TOL, cfg_and_prm  # noqa: E402


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_matches_eval_idos_twice(precision):
    w, cfg, prm = cfg_and_prm(precision=precision)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    with pkg.create_model(cfg) as m:
        # float64 matrices up to 2N^2 = 112 take the shared-memory path
        cases = ((4, 6, 3), (8, 3, 5)) if precision == "fp32" else ((4, 6, 3), (7, 2, 5))
        for N, K, sample in cases:
            ref_Q, ref_E = m.eval_idos(N, K, seed=w["seed"], level=1, sample=sample, want_eigs=True)
            for call in range(2):       # two calls in a row share the static scratch
                q = torch.full((w["n_E"],), float("nan"), dtype=torch.float64, device=dev)
                binding.eval_idos_noalloc(cfg, N, K, q.data_ptr(), seed=w["seed"], level=1, sample=sample,
                                          stream=stream)
                e = torch.full((K * K, 2 * N * N), float("nan"), dtype=torch.float64, device=dev)
                q2 = torch.empty_like(q)
                binding.eval_idos_noalloc(cfg, N, K, q2.data_ptr(), eigs_dev_ptr=e.data_ptr(), seed=w["seed"],
                                          level=1, sample=sample, stream=stream)
                torch.cuda.synchronize()
                Q = q.cpu().numpy()
                assert np.max(np.abs(Q - ref_Q)) < IDOS_TOL, (N, call)
                assert np.max(np.abs(q2.cpu().numpy() - ref_Q)) < IDOS_TOL, (N, call)
                E = e.cpu().numpy()
                assert np.array_equal(np.isnan(E), np.isnan(ref_E))
                ok = ~np.isnan(ref_E)
                assert np.max(np.abs(E[ok] - ref_E[ok])) < EIG_TOL


def test_noalloc_given_mask_and_limits():
    w, cfg, prm = cfg_and_prm(precision="fp32")
    dev = torch.device("cuda", 0)
    mask = np.zeros(32, np.uint8)
    mask[[1, 6, 17]] = 1
    with pkg.create_model(cfg) as m:
        ref = m.eval_idos(4, 2, mask=mask)
    md = torch.from_numpy(mask).to(dev)
    q = torch.empty(w["n_E"], dtype=torch.float64, device=dev)
    binding.eval_idos_noalloc(cfg, 4, 2, q.data_ptr(), mask_dev_ptr=md.data_ptr())
    torch.cuda.synchronize()
    assert np.max(np.abs(q.cpu().numpy() - ref)) < IDOS_TOL
    # beyond the shared-memory path and beyond the static scratch: clear errors
    with pytest.raises(pkg.IdosError) as ei:
        binding.eval_idos_noalloc(cfg, 16, 1, q.data_ptr())
    assert ei.value.status == -1
    with pytest.raises(pkg.IdosError) as ei:
        binding.eval_idos_noalloc(cfg, 8, 40, q.data_ptr())
    assert ei.value.status == -1 and "static scratch" in str(ei.value)


def test_noalloc_allocates_nothing_and_carries_no_state():
    """After a warm-up call (which may load the library's kernel modules), the
    device's free memory is the same before and after a series of calls,
    including a large call followed by a small one on the same scratch; the
    small call's result after the large one equals its result before it."""
    w, cfg, prm = cfg_and_prm(precision="fp32")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    small = torch.empty(w["n_E"], dtype=torch.float64, device=dev)
    large = torch.empty(w["n_E"], dtype=torch.float64, device=dev)
    again = torch.empty(w["n_E"], dtype=torch.float64, device=dev)
    e_small = torch.empty((4, 32), dtype=torch.float64, device=dev)
    binding.eval_idos_noalloc(cfg, 4, 2, small.data_ptr(), seed=w["seed"], level=0, sample=9, stream=stream)
    binding.eval_idos_noalloc(cfg, 8, 6, large.data_ptr(), seed=w["seed"], level=1, sample=9, stream=stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    for _ in range(3):
        binding.eval_idos_noalloc(cfg, 8, 6, large.data_ptr(), seed=w["seed"], level=1, sample=9, stream=stream)
        binding.eval_idos_noalloc(cfg, 4, 2, again.data_ptr(), eigs_dev_ptr=e_small.data_ptr(), seed=w["seed"],
                                  level=0, sample=9, stream=stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0, (free0, free1)
    assert torch.equal(small, again)
