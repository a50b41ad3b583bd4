"""The allocation-free G build agrees with the oracle and with the allocating one.

xs_gbuild_noalloc serves callers that cannot call cudaMalloc during the call:
a process whose device memory is reserved up front by another allocator's
pool, or a latency-critical loop that must not meet cudaMalloc's implicit
device synchronisation.  Its scratch is a fixed array inside the library.
Collected last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import molgen
from tests.gpu_common import rel_err

pytestmark = pytest.mark.gpu


def test_noalloc_gbuild_matches_oracle_and_xs_apply_twice():
    torch = pytest.importorskip("torch")
    from oracle import excited, nddo
    from paper_2505_24807_gb300 import xs
    params = molgen.make_params(0)
    Z, xyz = molgen.config_small(2)
    mol = nddo.Molecule(Z, xyz, params)
    ints = nddo.Integrals(mol)
    with xs.Context(0, molgen.params_table(params)) as ctx:
        xs.xs_ground_state(ctx, [(Z, xyz)])
        n, _, _ = xs.xs_get_sizes(ctx, 0)
        assert n == mol.nao
        rng = np.random.default_rng(11)
        for call in range(2):
            # fresh R on every call: the second call must not see the first's scratch
            R = rng.uniform(-1.0, 1.0, size=(3, n, n))
            oracle_G = excited.apply_kind(mol, ints, None, None, None, R, "G")
            ref = xs.xs_apply(ctx, 0, xs.XS_KIND_G, R)          # allocating path, host arrays
            R_dev = torch.from_numpy(R).cuda()
            G_dev = torch.full((3, n, n), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            xs.xs_gbuild_noalloc(ctx, 0, R_dev, G_dev)
            torch.cuda.synchronize()
            G = G_dev.cpu().numpy()
            # float64 throughout: only the rounding order differs from the oracle
            assert rel_err(G, oracle_G) < 1e-12, (call, rel_err(G, oracle_G))
            assert rel_err(G, ref) < 1e-12, (call, rel_err(G, ref))


def test_noalloc_gbuild_rejects_oversized_requests():
    torch = pytest.importorskip("torch")
    from paper_2505_24807_gb300 import xs
    params = molgen.make_params(0)
    Z, xyz = molgen.config_small(2)
    with xs.Context(0, molgen.params_table(params)) as ctx:
        xs.xs_ground_state(ctx, [(Z, xyz)])
        n, _, _ = xs.xs_get_sizes(ctx, 0)
        nvec = 2000   # 2 * nprod * nvec is beyond the 2^18-double scratch
        R_dev = torch.zeros((nvec, n, n), dtype=torch.float64, device="cuda")
        G_dev = torch.zeros_like(R_dev)
        with pytest.raises(xs.XSError) as e:
            xs.xs_gbuild_noalloc(ctx, 0, R_dev, G_dev)
        assert e.value.status == xs.XS_EINVAL
        # host pointers are refused too
        with pytest.raises(xs.XSError):
            xs.xs_gbuild_noalloc(ctx, 0, np.zeros((1, n, n)), np.zeros((1, n, n)))
