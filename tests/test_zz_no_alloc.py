"""The allocation-free residual entry point against the ordinary one.

stk_residual_norm_static serves callers that must not allocate device memory
while they run (a fixed memory budget, or a thread that must not block on
cudaMalloc); its scratch is a fixed static device array.  This file is named so
that pytest collects it last.  It checks, through the C ABI and on two calls in
a row (the second with different inputs, so stale scratch would show), that the
residual and its squared norm equal those of stk_residual within the 1e-12
relative tolerance the other FP64 tests use, and that the residual is the
oracle's b - A x to the same tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1911_05888_gb300 import problems as P  # noqa: E402
from paper_1911_05888_gb300.solver import StokesMG  # noqa: E402

pytestmark = pytest.mark.gpu


def test_static_scratch_residual_matches_allocating_entry_point():
    from oracle import multigrid
    prob = P.stress_variable_mu_2d(n=16, p=3)
    mg = StokesMG(prob)
    A = multigrid.Multigrid(prob).A
    rng = np.random.default_rng(17)
    b = torch.from_numpy(rng.uniform(-1, 1, prob.n_dofs)).cuda()
    for call in range(2):
        x = torch.from_numpy(rng.uniform(-1, 1, prob.n_dofs) * (call + 1)).cuda()
        r_ref = torch.empty_like(x)
        nrm_ref = mg.ctx.residual(x, b, r_ref, want_norm=True)
        r = torch.full_like(x, float("nan"))
        norm2 = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        mg.ctx.residual_norm_static(x, b, r, norm2)
        torch.cuda.synchronize()
        r_ref_h, r_h = r_ref.cpu().numpy(), r.cpu().numpy()
        assert np.linalg.norm(r_h - r_ref_h) <= 1e-12 * np.linalg.norm(r_ref_h)
        assert abs(np.sqrt(norm2.item()) - nrm_ref) <= 1e-12 * nrm_ref
        r_orc = b.cpu().numpy() - A @ x.cpu().numpy()
        assert np.linalg.norm(r_h - r_orc) <= 1e-12 * np.linalg.norm(r_orc)
    mg.close()
