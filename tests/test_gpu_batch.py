"""Batched persistent launch over many uneven matrices (graph replay), its
policies, configurations and autotuner, against the oracle and against each
member's own single-matrix kernels."""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import TOL_FP64, dev, host

pytestmark = pytest.mark.gpu

K = 4


def members(count=24, seed=0, integer=False):
    out = []
    for m in range(count):
        A = gen.powerlaw_batch_member(m, seed=seed, dim_lo=1e3, dim_hi=2e4)
        if integer:
            A.val = np.random.default_rng(m).integers(-1024, 1025, A.nnz).astype(np.float64)
        out.append(A)
    return out


def operands(As, k=K, integer=False, seed=1):
    rng = np.random.default_rng(seed)
    Bs = [(rng.integers(-1024, 1025, (A.n_cols, k)).astype(np.float64) if integer
           else gen.rhs_block(A.n_cols, k, seed=100 + i)) for i, A in enumerate(As)]
    return Bs


def run_batch(lib, As, Bs, policies=None, k=K, cfg=None, separate=False):
    import torch
    plans = [lib.Plan.from_csr(A) for A in As]
    Bd = [dev(B) for B in Bs]
    Cd = [torch.full((A.n_rows, k), float("nan"), dtype=torch.float64, device="cuda") for A in As]
    with lib.Batch(plans, k, policies) as b:
        if cfg:
            b.set_config(**cfg)
        b.set_io(Bd, Cd)
        (b.apply_separate if separate else b.apply)()
        torch.cuda.synchronize()
        out = [host(C) for C in Cd]
    for p in plans:
        p.close()
    return out


def check(As, Bs, Cs, exact=False):
    for A, B, C in zip(As, Bs, Cs):
        ref = oracle.spmm(A, B)
        if exact:
            assert np.array_equal(C, ref)
        else:
            assert oracle.max_err_ratio(C, ref, oracle.abs_scale(A, B), TOL_FP64) <= 1.0


@pytest.mark.parametrize("policy", ["l1", "l2", "l4", "l8", "l32", "adapt", "sorted", "mixed"])
def test_batch_matches_oracle(lib, policy):
    As = members()
    Bs = operands(As)
    if policy == "mixed":
        pol = [m % lib.SPMV_BATCH_N_POLICIES for m in range(len(As))]
    else:
        pol = [{v: k for k, v in lib.POLICY_NAMES.items()}[policy]] * len(As)
    check(As, Bs, run_batch(lib, As, Bs, pol))


def test_batch_integer_bit_exact(lib):
    As = members(12, integer=True)
    Bs = operands(As, integer=True)
    pol = [m % lib.SPMV_BATCH_N_POLICIES for m in range(len(As))]
    check(As, Bs, run_batch(lib, As, Bs, pol), exact=True)


@pytest.mark.parametrize("policy,variant", [(0, 2), (1, 3), (2, 4), (3, 5), (4, 7)])
def test_batch_equals_solo_kernel_bitwise(lib, policy, variant):
    """A member under a fixed-L policy sums each row in the same order as the
    single-matrix L-lanes kernel: the results agree bit for bit."""
    import torch
    As = members(6)
    Bs = operands(As)
    Cb = run_batch(lib, As, Bs, [policy] * len(As))
    for A, B, C in zip(As, Bs, Cb):
        with lib.Plan.from_csr(A, variant=variant) as p:
            Cs = torch.empty((A.n_rows, K), dtype=torch.float64, device="cuda")
            p.apply_block(dev(B), Cs)
            assert np.array_equal(host(Cs), C)


@pytest.mark.parametrize("cfg", [dict(item_nnz=64, schedule=0, ctas_per_sm=1),
                                 dict(item_nnz=4096, schedule=1, ctas_per_sm=8),
                                 dict(item_nnz=1 << 20, schedule=0, ctas_per_sm=4),
                                 dict(item_nnz=300, schedule=1, ctas_per_sm=2),
                                 dict(item_nnz=512, schedule=0, ctas_per_sm=8)])   # static, CTAs beyond residency
def test_batch_configs_same_result(lib, cfg):
    As = members(10)
    Bs = operands(As)
    for p in (lib.SPMV_BATCH_ADAPT, lib.SPMV_BATCH_SORTED):
        pol = [p] * len(As)
        base = run_batch(lib, As, Bs, pol)
        got = run_batch(lib, As, Bs, pol, cfg=cfg)
        for a, b in zip(base, got):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("k", [1, 2, 3, 8, 16])
@pytest.mark.parametrize("policy", ["adapt", "sorted"])
def test_batch_other_k(lib, k, policy):
    """Every width of the kernel (k = 1, 2, 4 for k = 3, 8, 16; each with its
    own register budget and resident CTAs) against the oracle."""
    As = members(8)
    Bs = operands(As, k=k)
    pol = lib.SPMV_BATCH_ADAPT if policy == "adapt" else lib.SPMV_BATCH_SORTED
    check(As, Bs, run_batch(lib, As, Bs, [pol] * len(As), k=k))


def test_batch_separate_launches(lib):
    As = members(8)
    Bs = operands(As)
    check(As, Bs, run_batch(lib, As, Bs, separate=True))


def test_batch_host_path(lib):
    """spmv_batch_apply_host: B from pinned host buffers into the batch's device
    B, the batched launch, C back to host buffers; the same bits as the device
    path, repeated steps with new inputs, and the refusal of padded blocks."""
    import torch
    As = members(12, seed=3)
    plans = [lib.Plan.from_csr(A) for A in As]
    Bd = [torch.zeros((A.n_cols, K), dtype=torch.float64, device="cuda") for A in As]
    Cd = [torch.full((A.n_rows, K), float("nan"), dtype=torch.float64, device="cuda") for A in As]
    stream = torch.cuda.Stream()
    with lib.Batch(plans, K) as b:
        b.set_io(Bd, Cd)
        for step in range(3):
            Bs = operands(As, seed=10 + step)
            Bpin = [torch.from_numpy(B).pin_memory() for B in Bs]
            Cpin = [torch.full((A.n_rows, K), float("nan"), dtype=torch.float64).pin_memory() for A in As]
            b.apply_host(Bpin, Cpin, stream)
            stream.synchronize()
            Ch = [C.numpy().copy() for C in Cpin]
            check(As, Bs, Ch)
            b.apply(stream)                      # device path on the B the host path left behind
            stream.synchronize()
            for Cdev, C in zip(Cd, Ch):
                assert np.array_equal(host(Cdev), C)
        # members back to back in one device and one pinned allocation: one copy per operand, same bits
        nb, nc = [A.n_cols * K for A in As], [A.n_rows * K for A in As]
        Bf = torch.zeros(sum(nb), dtype=torch.float64, device="cuda")
        Cf = torch.full((sum(nc),), float("nan"), dtype=torch.float64, device="cuda")
        b.set_io([v.view(A.n_cols, K) for v, A in zip(torch.split(Bf, nb), As)],
                 [v.view(A.n_rows, K) for v, A in zip(torch.split(Cf, nc), As)])
        Bh = torch.from_numpy(np.concatenate([B.ravel() for B in Bs])).pin_memory()
        Chf = torch.full((sum(nc),), float("nan"), dtype=torch.float64).pin_memory()
        b.apply_host(list(torch.split(Bh, nb)), list(torch.split(Chf, nc)), stream)
        stream.synchronize()
        for C, Cp in zip(Ch, torch.split(Chf, nc)):
            assert np.array_equal(Cp.numpy().reshape(C.shape), C)
        b.set_io(Bd, Cd)
        # a padded block (ld > k) cannot take the host path
        Bw = [torch.zeros((A.n_cols, K + 2), dtype=torch.float64, device="cuda") for A in As]
        b.set_io(Bw, Cd)
        with pytest.raises(lib.SpmvError) as e:
            b.apply_host(Bpin, Cpin, stream)
        assert e.value.status == 1
    for p in plans:
        p.close()


def test_batch_replay_autotune_and_new_io(lib):
    import torch
    As = members(16)
    Bs = operands(As)
    plans = [lib.Plan.from_csr(A) for A in As]
    Bd = [dev(B) for B in Bs]
    Cd = [torch.zeros((A.n_rows, K), dtype=torch.float64, device="cuda") for A in As]
    with lib.Batch(plans, K) as b:
        n_items, rows, nnz = b.info()
        assert rows == sum(A.n_rows for A in As) and nnz == sum(A.nnz for A in As) and n_items > len(As)
        b.set_io(Bd, Cd)
        for _ in range(3):
            b.apply()
        torch.cuda.synchronize()
        first = [host(C) for C in Cd]
        check(As, Bs, first)
        best, times = b.autotune(reps=2)
        assert len(times) == len(lib.AUTOTUNE_GRID) and np.all(times > 0)
        c = b.config()
        assert (c.item_nnz, c.schedule, c.ctas_per_sm) == (best.item_nnz, best.schedule, best.ctas_per_sm)
        Cd2 = [torch.full((A.n_rows, K), float("nan"), dtype=torch.float64, device="cuda") for A in As]
        b.set_io(Bd, Cd2)
        b.apply()
        torch.cuda.synchronize()
        for a, C in zip(first, Cd2):
            assert np.array_equal(a, host(C))
    for p in plans:
        p.close()


def test_batch_empty_members_and_errors(lib):
    import torch
    empty = gen.CSR(0, 10, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    blank = gen.CSR(50, 10, np.zeros(51, np.int32), np.zeros(0, np.int32), np.zeros(0))
    A = gen.powerlaw(3000, seed=2)
    As = [empty, blank, A]
    Bs = [gen.rhs_block(M.n_cols, K, seed=i) for i, M in enumerate(As)]
    Cs = run_batch(lib, As, Bs, [lib.SPMV_BATCH_ADAPT, lib.SPMV_BATCH_L1, lib.SPMV_BATCH_L32])
    assert Cs[0].shape == (0, K)
    assert np.array_equal(Cs[1], np.zeros((50, K)))
    check([A], [Bs[2]], [Cs[2]])
    with lib.Plan.from_csr(A) as p:
        for bad in (dict(k=0), dict(k=17), dict(k=4, policies=[9])):
            with pytest.raises(lib.SpmvError) as e:
                lib.Batch([p], bad["k"], bad.get("policies"))
            assert e.value.status == 1
        with lib.Batch([p], 4) as b:
            with pytest.raises(lib.SpmvError):
                b.apply()        # no operands set
            with pytest.raises(lib.SpmvError):
                b.set_config(item_nnz=1)
            with pytest.raises(lib.SpmvError):
                b.set_config(schedule=2)
            with pytest.raises(lib.SpmvError):
                b.set_io([dev(np.zeros((A.n_cols, 4)))], [torch.zeros((A.n_rows, 2), dtype=torch.float64,
                                                                        device="cuda")])


def test_set_io_waits_for_a_replay_on_a_non_blocking_stream(lib):
    """spmv_batch_set_io rewrites the device member table that a replay reads.
    A replay enqueued just before on a non-blocking stream (queued behind a
    busy kernel, so it has not started when set_io runs) must still see the
    operands it was enqueued with: set_io waits for it.  Both replays are
    checked against the oracle."""
    import torch
    As = members(16, seed=5)
    Bs1, Bs2 = operands(As, seed=21), operands(As, seed=22)
    plans = [lib.Plan.from_csr(A) for A in As]
    B1, B2 = [dev(B) for B in Bs1], [dev(B) for B in Bs2]
    C1 = [torch.full((A.n_rows, K), float("nan"), dtype=torch.float64, device="cuda") for A in As]
    C2 = [torch.full((A.n_rows, K), float("nan"), dtype=torch.float64, device="cuda") for A in As]
    s = torch.cuda.Stream()                      # non-blocking with respect to the legacy stream
    torch.cuda.synchronize()
    with lib.Batch(plans, K) as b:
        b.set_io(B1, C1)
        with torch.cuda.stream(s):
            torch.cuda._sleep(100_000_000)       # a bounded spin (about 50 ms) ahead of the replay
        b.apply(s)
        b.set_io(B2, C2)                         # returns only once the replay above has run
        b.apply(s)
        s.synchronize()
        check(As, Bs1, [host(C) for C in C1])
        check(As, Bs2, [host(C) for C in C2])
        # a member with nonzeros but no B is refused on the host
        with pytest.raises(lib.SpmvError) as e:
            lib.spmv_batch_set_io(b.handle, [0] * len(As), None, [C.data_ptr() for C in C1], None)
        assert e.value.status == 1 and "NULL B" in str(e.value)
    for p in plans:
        p.close()


def test_batch_host_async_pipeline(lib):
    """spmv_batch_apply_host_async: four pipelined steps with new page-locked
    operands each (copy-in of one step overlapping the launch and copy-out of
    its neighbours), members scattered over separate host buffers and members
    back to back in one; every step's C equals the oracle, bit for bit the
    device path's result on the same B."""
    import torch
    As = members(14, seed=6)
    plans = [lib.Plan.from_csr(A) for A in As]
    stream = torch.cuda.Stream()
    steps = [operands(As, seed=30 + i) for i in range(4)]
    with lib.Batch(plans, K) as b:
        pinB = [[torch.from_numpy(B).pin_memory() for B in Bs] for Bs in steps]
        pinC = [[torch.full((A.n_rows, K), float("nan"), dtype=torch.float64).pin_memory() for A in As]
                for _ in steps]
        for i in range(len(steps)):
            b.apply_host_async(pinB[i], pinC[i], stream)
        b.host_sync()
        for Bs, Cs in zip(steps, pinC):
            check(As, Bs, [C.numpy() for C in Cs])
        # the same products through the device path agree bit for bit
        Bd = [dev(B) for B in steps[2]]
        Cd = [torch.full((A.n_rows, K), float("nan"), dtype=torch.float64, device="cuda") for A in As]
        b.set_io(Bd, Cd)
        b.apply(stream)
        stream.synchronize()
        for C, Cp in zip(Cd, pinC[2]):
            assert np.array_equal(host(C), Cp.numpy())
        # members back to back in one pinned allocation (merged copies), after a configuration change
        b.set_config(item_nnz=512)
        nb, nc = [A.n_cols * K for A in As], [A.n_rows * K for A in As]
        Bf = torch.from_numpy(np.concatenate([B.ravel() for B in steps[3]])).pin_memory()
        Cf = torch.full((sum(nc),), float("nan"), dtype=torch.float64).pin_memory()
        b.apply_host_async(list(torch.split(Bf, nb)), list(torch.split(Cf, nc)), stream)
        b.host_sync()
        for C, Cp in zip(pinC[3], torch.split(Cf, nc)):
            assert np.array_equal(Cp.numpy().reshape(C.shape), C.numpy())
    for p in plans:
        p.close()
