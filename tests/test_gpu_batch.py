"""Operation-level batching: a plan of mixed NTT / INTT / HMULT operations of uneven ring
degree and level gives exactly the results of the single-operation calls, eagerly and when
replayed as one CUDA graph, in both plan modes (the persistent launch with its device work
queue, and the grouped launches); the persistent kernel's bounded dependency wait reports an
expired wait without hanging."""
import numpy as np
import pytest

from oracle import ckks as C
from oracle import ntt as ON
from oracle import params as P
from paper_2212_14191_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fhe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_14191_gb300 import fhe as f
    return f


def make_ops(fhe, qs, ps, seed):
    """Mixed list: NTT/INTT at N = 2^12..2^14 over varying limb ranges, HMULT at 2^12/2^13."""
    import torch
    g = np.random.default_rng(seed)
    mods = qs + ps
    ops, keep = [], []
    evks = {}
    for logn in (12, 13):
        dnum = -(-len(qs) // 4)
        evks[logn] = fhe.to_device(I.uniform_residues(seed + logn, mods, 2 * dnum, 1 << logn).reshape(
            len(mods), dnum, 2, 1 << logn).transpose(1, 2, 0, 3).copy())
    for i in range(14):
        kind = [fhe.FHE_OPK_NTT_FWD, fhe.FHE_OPK_NTT_INV, fhe.FHE_OPK_HMULT][i % 3]
        if kind == fhe.FHE_OPK_HMULT:
            logn = int(g.choice([12, 13]))
            nl, batch = int(g.integers(2, len(qs) + 1)), int(g.integers(1, 3))
            n = 1 << logn
            a = fhe.to_device(I.uniform_residues(seed + 100 + i, qs[:nl], 2 * batch, n).reshape(
                nl, 2, batch, n).transpose(1, 0, 2, 3).copy())
            b = fhe.to_device(I.uniform_residues(seed + 200 + i, qs[:nl], 2 * batch, n).reshape(
                nl, 2, batch, n).transpose(1, 0, 2, 3).copy())
            out = torch.empty((2, nl - 1, batch, n), dtype=torch.int32, device="cuda")
            ops.append(fhe.FheOp(kind=kind, logN=logn, first_limb=0, n_limbs=nl, batch=batch,
                                 a=a.data_ptr(), b=b.data_ptr(), evk=evks[logn].data_ptr(), out=out.data_ptr()))
            keep.append(("hmult", logn, nl, batch, a, b, evks[logn], out))
        else:
            logn = int(g.choice([12, 13, 14]))
            first = int(g.integers(0, len(mods) - 1))
            nl = int(g.integers(1, len(mods) - first + 1))
            batch = int(g.integers(1, 4))
            x = I.uniform_residues(seed + 300 + i, mods[first:first + nl], batch, 1 << logn)
            d = fhe.to_device(x)
            ops.append(fhe.FheOp(kind=kind, logN=logn, first_limb=first, n_limbs=nl, batch=batch,
                                 data=d.data_ptr()))
            keep.append(("ntt", logn, first, nl, batch, d, x, kind))
    return ops, keep


def reference_results(fhe, ctx, keep):
    import torch
    res = []
    for k in keep:
        if k[0] == "hmult":
            _, logn, nl, batch, a, b, evk, out = k
            res.append(fhe.to_host(ctx.hmult(a, b, evk, logn)))
        else:
            _, logn, first, nl, batch, d, x, kind = k
            t = fhe.to_device(x)
            if kind == fhe.FHE_OPK_NTT_FWD:
                ctx.ntt_fwd(t, logn, first_limb=first)
            else:
                ctx.ntt_inv(t, logn, first_limb=first)
            res.append(fhe.to_host(t))
    torch.cuda.synchronize()
    return res


def batch_results(fhe, keep):
    return [fhe.to_host(k[7] if k[0] == "hmult" else k[5]) for k in keep]


def reset_inputs(fhe, keep):
    for k in keep:
        if k[0] == "ntt":
            k[5].copy_(fhe.to_device(k[6]))


MODES = ["persistent", "grouped"]


def create(fhe, ctx, ops, mode, slot_bytes=0):
    m = fhe.FHE_BATCH_PERSISTENT if mode == "persistent" else fhe.FHE_BATCH_GROUPED
    return fhe.fhe_batch_create_ex(ctx.handle, ops, m, slot_bytes)


@pytest.mark.parametrize("mode", MODES)
def test_batch_equals_single_calls(fhe, mode):
    """N = 2^12..2^14: in persistent mode the 2^14 transforms run in the persistent launch and
    the smaller operations in grouped launches before it, in one plan."""
    import torch
    qs, ps = P.default_moduli(8, 4)
    ctx = fhe.Context(14, qs, ps, alpha=4)
    ops, keep = make_ops(fhe, qs, ps, 7)
    want = reference_results(fhe, ctx, keep)
    plan = create(fhe, ctx, ops, mode)
    nbytes = fhe.fhe_batch_scratch_bytes(plan)
    scratch = torch.empty(max(4, nbytes // 4 + 4), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    fhe.fhe_batch_run(plan, scratch.data_ptr(), nbytes, stream)
    torch.cuda.synchronize()
    got = batch_results(fhe, keep)
    for w, g in zip(want, got):
        assert (w == g).all()
    # one NTT op against the oracle directly
    for k, g in zip(keep, got):
        if k[0] == "ntt" and k[7] == fhe.FHE_OPK_NTT_FWD:
            _, logn, first, nl, batch, d, x, kind = k
            mods = (qs + ps)[first:first + nl]
            ref, _ = ON.ntt_batch(x, mods, [P.psi(m, 1 << logn) for m in mods])
            assert (g == ref).all()
            break
    # graph capture and two replays
    reset_inputs(fhe, keep)
    fhe.fhe_batch_capture(plan, scratch.data_ptr(), nbytes)   # runs once, then captures
    for _ in range(2):
        reset_inputs(fhe, keep)
        fhe.fhe_batch_launch(plan, stream)
        torch.cuda.synchronize()
        for w, g in zip(want, batch_results(fhe, keep)):
            assert (w == g).all()
    fhe.fhe_device_status(ctx.handle, 1)
    fhe.fhe_batch_destroy(plan)
    ctx.close()


def test_batch_hmult_matches_oracle(fhe):
    import torch
    qs, ps = P.default_moduli(8, 4)
    logn, n = 12, 1 << 12
    prm = C.Params(n, qs, ps, alpha=4)
    evk_h = I.uniform_residues(5, qs + ps, 2 * prm.dnum(8), n).reshape(12, prm.dnum(8), 2, n).transpose(1, 2, 0, 3).copy()
    evk = fhe.to_device(evk_h)
    ctx = fhe.Context(logn, qs, ps, alpha=4)
    ops, cts = [], []
    for i, nl in enumerate((3, 3, 6)):
        a = I.uniform_residues(40 + i, qs[:nl], 2, n).reshape(nl, 2, 1, n).transpose(1, 0, 2, 3).copy()
        b = I.uniform_residues(50 + i, qs[:nl], 2, n).reshape(nl, 2, 1, n).transpose(1, 0, 2, 3).copy()
        da, db = fhe.to_device(a), fhe.to_device(b)
        out = torch.empty((2, nl - 1, 1, n), dtype=torch.int32, device="cuda")
        ops.append(fhe.FheOp(kind=fhe.FHE_OPK_HMULT, logN=logn, n_limbs=nl, batch=1, a=da.data_ptr(),
                             b=db.data_ptr(), evk=evk.data_ptr(), out=out.data_ptr()))
        cts.append((nl, a, b, da, db, out))
    plan = fhe.fhe_batch_create(ctx.handle, ops)
    nbytes = fhe.fhe_batch_scratch_bytes(plan)
    scratch = torch.empty(nbytes // 4 + 4, dtype=torch.int32, device="cuda")
    fhe.fhe_batch_run(plan, scratch.data_ptr(), nbytes, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for nl, a, b, _, _, out in cts:
        want = C.hmult(prm, nl, a[:, :, 0].astype(np.uint64), b[:, :, 0].astype(np.uint64), evk_h.astype(np.uint64))
        assert (fhe.to_host(out)[:, :, 0] == want).all()
    fhe.fhe_batch_destroy(plan)
    ctx.close()


def test_batch_rejects_bad_ops(fhe):
    qs, ps = P.default_moduli(4, 2)
    ctx = fhe.Context(12, qs, ps, alpha=2)
    for op in (fhe.FheOp(kind=9, logN=12, n_limbs=1, batch=1, data=16),
               fhe.FheOp(kind=fhe.FHE_OPK_NTT_FWD, logN=13, n_limbs=1, batch=1, data=16),
               fhe.FheOp(kind=fhe.FHE_OPK_NTT_FWD, logN=12, first_limb=5, n_limbs=2, batch=1, data=16),
               fhe.FheOp(kind=fhe.FHE_OPK_HMULT, logN=12, n_limbs=1, batch=1, a=16, b=16, evk=16, out=16)):
        with pytest.raises(fhe.FheError) as e:
            fhe.fhe_batch_create(ctx.handle, [op])
        assert e.value.code == fhe.FHE_EINVAL
    ctx.close()


@pytest.mark.parametrize("mode", MODES)
def test_batch_full_size_ring_degrees(fhe, mode):
    """A plan at the uneven-batch workload's sizes: NTT and INTT rows at N = 2^15 and 2^16 with
    24 to 44 limbs (the two-pass row-table kernels) and HMULT groups at 2^15 and 2^16 with 24,
    36 and 44 limbs (3, 5 and 6 key-switching slices; one group gathers two operations). Every
    operation equals its single call, eagerly and after graph capture; sampled NTT rows and
    one 44-limb HMULT are compared with the oracle."""
    import torch
    qs, ps = P.default_moduli(44, 8)
    mods = qs + ps
    ctx = fhe.Context(16, qs, ps, alpha=8)
    prm = {lg: C.Params(1 << lg, qs, ps, alpha=8) for lg in (15, 16)}
    evk_h, evks = {}, {}
    for lg in (15, 16):
        n = 1 << lg
        dn = prm[lg].dnum(len(qs))
        evk_h[lg] = I.uniform_residues(900 + lg, mods, 2 * dn, n).reshape(len(mods), dn, 2, n).transpose(1, 2, 0, 3).copy()
        evks[lg] = fhe.to_device(evk_h[lg])
    ops, keep = [], []
    ntt_specs = [(16, fhe.FHE_OPK_NTT_FWD, 0, 24, 2), (15, fhe.FHE_OPK_NTT_INV, 0, 44, 1),
                 (15, fhe.FHE_OPK_NTT_FWD, 8, 30, 2), (16, fhe.FHE_OPK_NTT_INV, 4, 40, 1),
                 (16, fhe.FHE_OPK_NTT_FWD, 44, 8, 1)]
    for i, (lg, kind, first, nl, batch) in enumerate(ntt_specs):
        x = I.uniform_residues(950 + i, mods[first:first + nl], batch, 1 << lg)
        d = fhe.to_device(x)
        ops.append(fhe.FheOp(kind=kind, logN=lg, first_limb=first, n_limbs=nl, batch=batch, data=d.data_ptr()))
        keep.append(("ntt", lg, first, nl, batch, d, x, kind))
    hm_specs = [(16, 44, 1), (15, 36, 1), (15, 36, 2), (16, 24, 1)]
    for i, (lg, nl, batch) in enumerate(hm_specs):
        n = 1 << lg
        a = fhe.to_device(I.uniform_residues(970 + i, qs[:nl], 2 * batch, n).reshape(nl, 2, batch, n).transpose(1, 0, 2, 3).copy())
        b = fhe.to_device(I.uniform_residues(980 + i, qs[:nl], 2 * batch, n).reshape(nl, 2, batch, n).transpose(1, 0, 2, 3).copy())
        out = torch.empty((2, nl - 1, batch, n), dtype=torch.int32, device="cuda")
        ops.append(fhe.FheOp(kind=fhe.FHE_OPK_HMULT, logN=lg, n_limbs=nl, batch=batch, a=a.data_ptr(),
                             b=b.data_ptr(), evk=evks[lg].data_ptr(), out=out.data_ptr()))
        keep.append(("hmult", lg, nl, batch, a, b, evks[lg], out))
    want = reference_results(fhe, ctx, keep)
    plan = create(fhe, ctx, ops, mode)
    nbytes = fhe.fhe_batch_scratch_bytes(plan)
    scratch = torch.empty(max(4, nbytes // 4 + 4), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    fhe.fhe_batch_run(plan, scratch.data_ptr(), nbytes, stream)
    torch.cuda.synchronize()
    got = batch_results(fhe, keep)
    for i, (w, g) in enumerate(zip(want, got)):
        assert (w == g).all(), i
    # oracle: the first and last limb of every NTT op (first polynomial), and the 44-limb HMULT
    for k, g in zip(keep, got):
        if k[0] == "ntt":
            _, lg, first, nl, batch, d, x, kind = k
            for l in (0, nl - 1):
                m = mods[first + l]
                ref, _ = ON.ntt_batch(x[l:l + 1, :1], [m], [P.psi(m, 1 << lg)], inverse=kind == fhe.FHE_OPK_NTT_INV)
                assert (g[l:l + 1, :1] == ref).all(), (lg, first, l)
    _, lg, nl, batch, a, b, evk, out = keep[len(ntt_specs)]
    ha, hb = fhe.to_host(a), fhe.to_host(b)
    oracle = C.hmult(prm[lg], nl, ha[:, :, 0].astype(np.uint64), hb[:, :, 0].astype(np.uint64),
                     evk_h[lg].astype(np.uint64))
    assert (got[len(ntt_specs)][:, :, 0] == oracle).all()
    # graph capture and a replay
    reset_inputs(fhe, keep)
    fhe.fhe_batch_capture(plan, scratch.data_ptr(), nbytes)
    reset_inputs(fhe, keep)
    fhe.fhe_batch_launch(plan, stream)
    torch.cuda.synchronize()
    for i, (w, g) in enumerate(zip(want, batch_results(fhe, keep))):
        assert (w == g).all(), i
    fhe.fhe_device_status(ctx.handle, 1)
    fhe.fhe_batch_destroy(plan)
    ctx.close()


@pytest.mark.parametrize("slot_bytes", [1, 0])
def test_persistent_hmult_slots(fhe, slot_bytes):
    """Persistent mode with HMULTs at N = 2^14, 2^15 and 2^16 (3 to 24 limbs, batches of one and
    two ciphertexts) between NTT and INTT operations. slot_bytes = 1 leaves one scratch slot, so
    every HMULT waits for the one before it (the chained dependency); 0 gives each HMULT its own
    slot. Every result equals the single call, on the eager run and on two graph replays with
    the inputs restored in between; one HMULT per ring degree is compared with the oracle."""
    import torch
    qs, ps = P.default_moduli(24, 8)
    mods = qs + ps
    ctx = fhe.Context(16, qs, ps, alpha=8)
    evk_h, evks, prm = {}, {}, {}
    for lg in (14, 15, 16):
        n = 1 << lg
        prm[lg] = C.Params(n, qs, ps, alpha=8)
        dn = prm[lg].dnum(len(qs))
        evk_h[lg] = I.uniform_residues(1200 + lg, mods, 2 * dn, n).reshape(len(mods), dn, 2, n).transpose(1, 2, 0, 3).copy()
        evks[lg] = fhe.to_device(evk_h[lg])
    ops, keep = [], []
    specs = [("hmult", 16, 24, 1), ("ntt", 15, 0, 12, 2, fhe.FHE_OPK_NTT_FWD), ("hmult", 14, 3, 2),
             ("hmult", 15, 17, 1), ("ntt", 14, 3, 20, 1, fhe.FHE_OPK_NTT_INV), ("hmult", 16, 9, 2),
             ("hmult", 14, 24, 1), ("ntt", 16, 30, 2, 1, fhe.FHE_OPK_NTT_INV)]
    for i, sp in enumerate(specs):
        if sp[0] == "hmult":
            _, lg, nl, batch = sp
            n = 1 << lg
            a = fhe.to_device(I.uniform_residues(1300 + i, qs[:nl], 2 * batch, n).reshape(nl, 2, batch, n).transpose(1, 0, 2, 3).copy())
            b = fhe.to_device(I.uniform_residues(1400 + i, qs[:nl], 2 * batch, n).reshape(nl, 2, batch, n).transpose(1, 0, 2, 3).copy())
            out = torch.full((2, nl - 1, batch, n), -1, dtype=torch.int32, device="cuda")
            ops.append(fhe.FheOp(kind=fhe.FHE_OPK_HMULT, logN=lg, n_limbs=nl, batch=batch, a=a.data_ptr(),
                                 b=b.data_ptr(), evk=evks[lg].data_ptr(), out=out.data_ptr()))
            keep.append(("hmult", lg, nl, batch, a, b, evks[lg], out))
        else:
            _, lg, first, nl, batch, kind = sp
            x = I.uniform_residues(1500 + i, mods[first:first + nl], batch, 1 << lg)
            d = fhe.to_device(x)
            ops.append(fhe.FheOp(kind=kind, logN=lg, first_limb=first, n_limbs=nl, batch=batch, data=d.data_ptr()))
            keep.append(("ntt", lg, first, nl, batch, d, x, kind))
    want = reference_results(fhe, ctx, keep)
    plan = create(fhe, ctx, ops, "persistent", slot_bytes)
    nbytes = fhe.fhe_batch_scratch_bytes(plan)
    scratch = torch.full((nbytes // 4 + 4,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    fhe.fhe_batch_run(plan, scratch.data_ptr(), nbytes, stream)
    torch.cuda.synchronize()
    fhe.fhe_device_status(ctx.handle, 1)
    got = batch_results(fhe, keep)
    for i, (w, g) in enumerate(zip(want, got)):
        assert (w == g).all(), (i, specs[i])
    seen = set()
    for k, g in zip(keep, got):
        if k[0] == "hmult" and k[1] not in seen:
            seen.add(k[1])
            _, lg, nl, batch, a, b, evk, out = k
            ha, hb = fhe.to_host(a), fhe.to_host(b)
            oracle = C.hmult(prm[lg], nl, ha[:, :, batch - 1].astype(np.uint64), hb[:, :, batch - 1].astype(np.uint64),
                             evk_h[lg].astype(np.uint64))
            assert (g[:, :, batch - 1] == oracle).all(), (lg, nl)
    reset_inputs(fhe, keep)
    fhe.fhe_batch_capture(plan, scratch.data_ptr(), nbytes)
    for _ in range(2):
        reset_inputs(fhe, keep)
        for k in keep:
            if k[0] == "hmult":
                k[7].fill_(-1)
        fhe.fhe_batch_launch(plan, stream)
        torch.cuda.synchronize()
        fhe.fhe_device_status(ctx.handle, 1)
        for i, (w, g) in enumerate(zip(want, batch_results(fhe, keep))):
            assert (w == g).all(), (i, specs[i])
    fhe.fhe_batch_destroy(plan)
    ctx.close()


def test_persistent_queue_wait_expires(fhe):
    """The persistent kernel's dependency wait on a counter that nothing increments gives up
    after its cycle limit, records FHE_ETIMEOUT in the context's status word and ends; the
    context then runs a persistent plan correctly."""
    import torch
    qs, ps = P.default_moduli(4, 2)
    ctx = fhe.Context(14, qs, ps, alpha=2)
    fhe.fhe_selftest_queue_timeout(ctx.handle, 2_000_000, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    with pytest.raises(fhe.FheError) as e:
        fhe.fhe_device_status(ctx.handle, 1)
    assert e.value.code == fhe.FHE_ETIMEOUT
    fhe.fhe_device_status(ctx.handle, 1)          # cleared
    x = I.uniform_residues(1600, qs, 2, 1 << 14)
    d = fhe.to_device(x)
    plan = create(fhe, ctx, [fhe.FheOp(kind=fhe.FHE_OPK_NTT_FWD, logN=14, first_limb=0, n_limbs=len(qs), batch=2,
                                       data=d.data_ptr())], "persistent")
    nbytes = fhe.fhe_batch_scratch_bytes(plan)
    scratch = torch.empty(max(4, nbytes // 4 + 4), dtype=torch.int32, device="cuda")
    fhe.fhe_batch_run(plan, scratch.data_ptr(), nbytes, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    fhe.fhe_device_status(ctx.handle, 1)
    ref, _ = ON.ntt_batch(x, qs, [P.psi(q, 1 << 14) for q in qs])
    assert (fhe.to_host(d) == ref).all()
    fhe.fhe_batch_destroy(plan)
    ctx.close()


def _extreme(mods, count, n, kind):
    """(len(mods), count, n) uint32 residues: all q - 1 ("max") or q - 1 and 0 alternating."""
    q = np.array(mods, dtype=np.uint64)[:, None, None]
    x = np.broadcast_to(q - 1, (len(mods), count, n)).copy()
    if kind == "alt":
        x[:, :, 1::2] = 0
    return x.astype(np.uint32)


@pytest.mark.parametrize("mode", MODES)
def test_batch_extreme_residues(fhe, mode):
    """A plan at N = 2^14..2^16 whose operands and keys sit at the ends of their residue ranges
    (all q - 1, or q - 1 and 0 alternating): NTT and INTT rows and HMULTs through the persistent
    engine's stage bodies (and the grouped launches) equal their single calls, and one HMULT
    equals the oracle's."""
    import torch
    qs, ps = P.default_moduli(12, 4)
    mods = qs + ps
    ctx = fhe.Context(16, qs, ps, alpha=4)
    dn = -(-len(qs) // 4)
    evk_h = {lg: _extreme(mods, 2 * dn, 1 << lg, "max").reshape(len(mods), dn, 2, 1 << lg).transpose(1, 2, 0, 3).copy()
             for lg in (15, 16)}
    evks = {lg: fhe.to_device(e) for lg, e in evk_h.items()}
    ops, keep = [], []
    for lg, kind, first, nl, batch, pat in ((16, fhe.FHE_OPK_NTT_FWD, 0, 6, 2, "max"),
                                            (15, fhe.FHE_OPK_NTT_INV, 2, 8, 1, "alt"),
                                            (14, fhe.FHE_OPK_NTT_FWD, 10, 6, 3, "alt"),
                                            (16, fhe.FHE_OPK_NTT_INV, 0, 16, 1, "max")):
        x = _extreme(mods[first:first + nl], batch, 1 << lg, pat)
        d = fhe.to_device(x)
        ops.append(fhe.FheOp(kind=kind, logN=lg, first_limb=first, n_limbs=nl, batch=batch, data=d.data_ptr()))
        keep.append(("ntt", lg, first, nl, batch, d, x, kind))
    hm = []
    for lg, nl, batch in ((16, 6, 2), (15, 9, 1)):
        n = 1 << lg
        a_h = np.stack([_extreme(qs[:nl], batch, n, "max"), _extreme(qs[:nl], batch, n, "alt")])
        b_h = np.stack([_extreme(qs[:nl], batch, n, "alt"), _extreme(qs[:nl], batch, n, "max")])
        a, b = fhe.to_device(a_h), fhe.to_device(b_h)
        out = torch.empty((2, nl - 1, batch, n), dtype=torch.int32, device="cuda")
        ops.append(fhe.FheOp(kind=fhe.FHE_OPK_HMULT, logN=lg, n_limbs=nl, batch=batch, a=a.data_ptr(),
                             b=b.data_ptr(), evk=evks[lg].data_ptr(), out=out.data_ptr()))
        keep.append(("hmult", lg, nl, batch, a, b, evks[lg], out))
        hm.append((lg, nl, a_h, b_h))
    want = reference_results(fhe, ctx, keep)
    plan = create(fhe, ctx, ops, mode)
    nbytes = fhe.fhe_batch_scratch_bytes(plan)
    scratch = torch.empty(max(4, nbytes // 4 + 4), dtype=torch.int32, device="cuda")
    fhe.fhe_batch_run(plan, scratch.data_ptr(), nbytes, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = batch_results(fhe, keep)
    for i, (w, g) in enumerate(zip(want, got)):
        assert (w == g).all(), i
    lg, nl, a_h, b_h = hm[0]
    prm = C.Params(1 << lg, qs, ps, alpha=4)
    oracle = C.hmult(prm, nl, a_h[:, :, 0].astype(np.uint64), b_h[:, :, 0].astype(np.uint64),
                     evk_h[lg].astype(np.uint64))
    assert (got[len(keep) - 2][:, :, 0] == oracle).all()
    fhe.fhe_device_status(ctx.handle, 1)
    fhe.fhe_batch_destroy(plan)
    ctx.close()
