"""The allocation-free fused H_eff psi entry point (dmrg_hpsi_contract_noalloc)
against the allocating one (dmrg_hpsi_contract): same kernels and task
lists, so two calls in a row must give identical results.  The entry exists
for callers that must not allocate device memory while they run (a latency
loop where cudaMalloc would synchronise the device, or memory owned by
another allocator), so the free device memory must not change across a
warmed-up call.  Collected last so that it also runs after every other test
has used the device."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _problem(rng, n_blocks, max_dim, max_items):
    """Random sector-block contraction: ragged sizes, transposes, identities."""
    A_parts, P_parts, B_parts = [], [], []
    ao = po = bo = co = 0
    blocks, items = [], []
    for _ in range(n_blocks):
        m = int(rng.integers(1, max_dim))
        n = int(rng.integers(1, max_dim))
        ib = len(items)
        for _ in range(int(rng.integers(1, max_items + 1))):
            a_id = int(rng.random() < 0.15)
            b_id = int(rng.random() < 0.15) if not a_id else 0
            ka = m if a_id else int(rng.integers(1, max_dim))
            kb = n if b_id else int(rng.integers(1, max_dim))
            ta, tb = int(rng.integers(0, 2)), int(rng.integers(0, 2))
            if a_id:
                a_entry = (0, 1, 0)
            else:
                a = rng.standard_normal((ka, m) if ta else (m, ka))
                a_entry = (ao, a.shape[1], ta)
                A_parts.append(a.ravel())
                ao += a.size
            if b_id:
                b_entry = (0, 1, 0)
            else:
                b = rng.standard_normal((kb, n) if tb else (n, kb))
                b_entry = (bo, b.shape[1], tb)
                B_parts.append(b.ravel())
                bo += b.size
            Pm = rng.standard_normal((ka, kb))
            items.append((a_entry[0], po, b_entry[0], a_entry[1], kb, b_entry[1], a_entry[2],
                          b_entry[2], ka, kb, a_id, b_id, float(rng.standard_normal())))
            P_parts.append(Pm.ravel())
            po += Pm.size
        blocks.append((co, m, n, n, ib, len(items) - ib))
        co += m * n
    cat = lambda v: np.concatenate(v) if v else np.zeros(1)
    return cat(A_parts), cat(P_parts), cat(B_parts), co, blocks, items


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_allocating_entry_on_two_calls(precision):
    torch = pytest.importorskip("torch")
    import paper_2503_20700_gb300 as p
    p.load()
    rng = np.random.default_rng(21)
    A, P, B, clen, blocks, items = _problem(rng, 10, 140, 40)
    C0 = rng.standard_normal(clen)
    dev = torch.device("cuda:0")
    tA, tP, tB = (torch.from_numpy(x).to(dev) for x in (A, P, B))
    tC = torch.from_numpy(C0.copy()).to(dev)
    C_ref = C0.copy()
    stream = torch.cuda.current_stream(dev).cuda_stream
    for call in range(2):
        p.ops.hpsi_contract(A, P, B, C_ref, blocks, items, precision=precision)
        p.ops.hpsi_contract_noalloc(tA.data_ptr(), A.size, tP.data_ptr(), P.size, tB.data_ptr(), B.size,
                                    tC.data_ptr(), clen, blocks, items, precision=precision,
                                    device=0, stream=stream)
        torch.cuda.synchronize(dev)
        got = tC.cpu().numpy()
        assert np.array_equal(got, C_ref), f"call {call}: max diff {np.abs(got - C_ref).max()}"


def test_noalloc_rejects_oversize_and_bad_offsets():
    torch = pytest.importorskip("torch")
    import paper_2503_20700_gb300 as p
    p.load()
    dev = torch.device("cuda:0")
    # 8 blocks of 512 x 512 with 40 items each: thousands of partial tiles
    m = 512
    blocks = [(b * m * m, m, m, m, 40 * b, 40) for b in range(8)]
    items = [(0, 0, 0, 1, m, 1, 0, 0, m, m, 1, 1, 1.0)] * 320
    t = torch.zeros(8 * m * m, dtype=torch.float64, device=dev)
    with pytest.raises(p.DmrgError) as ei:
        p.ops.hpsi_contract_noalloc(t.data_ptr(), 1, t.data_ptr(), t.numel(), t.data_ptr(), 1,
                                    t.data_ptr(), t.numel(), blocks, items, precision=0)
    assert ei.value.status == p.DMRG_EINVAL and "scratch" in str(ei.value)
    bad = [(0, 10, 0, 4, 4, 4, 0, 0, 4, 4, 0, 0, 1.0)]
    with pytest.raises(p.DmrgError) as ei:
        p.ops.hpsi_contract_noalloc(t.data_ptr(), 4, t.data_ptr(), 4, t.data_ptr(), 4,
                                    t.data_ptr(), 16, [(0, 4, 4, 4, 0, 1)], bad, precision=0)
    assert ei.value.status == p.DMRG_EINVAL


def _near_limit_problem(rng, items_per_block):
    """One 512 x 512 sigma block of identity-left items (alpha P op(B)^T):
    the float64 kernel plans 64 x 64 tiles in item chunks of 4, so 60 items
    need 64 tiles x 15 chunks = 960 partial tiles (31.5 MB with the task
    lists, just under the 32 MiB scratch) and 64 items need 1024 (over it)."""
    m, kb = 512, 16
    P = rng.standard_normal(m * kb)
    B = rng.standard_normal(m * kb)
    items = [(0, 0, 0, 1, kb, kb, 0, 0, m, kb, 1, 0, float(rng.standard_normal()))
             for _ in range(items_per_block)]
    return P, B, m, [(0, m, m, m, 0, items_per_block)], items


def test_noalloc_near_capacity_and_no_device_allocation():
    torch = pytest.importorskip("torch")
    import paper_2503_20700_gb300 as p
    p.load()
    rng = np.random.default_rng(5)
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev).cuda_stream
    P, B, m, blocks, items = _near_limit_problem(rng, 60)
    A = np.zeros(1)
    C0 = rng.standard_normal(m * m)
    tA, tP, tB = (torch.from_numpy(x).to(dev) for x in (A, P, B))
    tC = torch.from_numpy(C0.copy()).to(dev)
    C_ref = C0.copy()

    def call():
        p.ops.hpsi_contract_noalloc(tA.data_ptr(), A.size, tP.data_ptr(), P.size, tB.data_ptr(), B.size,
                                    tC.data_ptr(), m * m, blocks, items, precision=0, device=0,
                                    stream=stream)
        torch.cuda.synchronize(dev)

    call()  # first call on the device: module load and symbol lookup
    p.ops.hpsi_contract(A, P, B, C_ref, blocks, items, precision=0)
    assert np.array_equal(tC.cpu().numpy(), C_ref)
    free0, _ = torch.cuda.mem_get_info(dev)
    call()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
    p.ops.hpsi_contract(A, P, B, C_ref, blocks, items, precision=0)
    assert np.array_equal(tC.cpu().numpy(), C_ref)
    # four more items push the partial tiles past the scratch
    _, _, _, blocks2, items2 = _near_limit_problem(rng, 64)
    with pytest.raises(p.DmrgError) as ei:
        p.ops.hpsi_contract_noalloc(tA.data_ptr(), A.size, tP.data_ptr(), P.size, tB.data_ptr(), B.size,
                                    tC.data_ptr(), m * m, blocks2, items2, precision=0, device=0,
                                    stream=stream)
    assert ei.value.status == p.DMRG_EINVAL and "scratch" in str(ei.value)
