"""The timed workloads at full size, in the launch configuration the benchmark
times (its own push loops: bench.Runner and bench.PushRun, pushes of 8192
samples on device pointers, then the flush), sampled outputs against the FP64
oracle one by one (Eq. 4 at each output).

  multi   64 streams x 480000 samples, own IRs L = 48000 swapped every 24000
          samples (20 versions), block 128: K1
  shared  1024 streams x 240000 samples, one IR L = 96000, block 256: K2
          (BF16 split, BF16) and K1 (FP32)
  mimo    16 x 16, 60 s per input, L = 192000, block 512: K3 (BF16 split, BF16)
          and K1 (FP32)
"""
import numpy as np
import pytest

import bench
import oracle
from gpu_helpers import TOL, rel_l2
from paper_2401_01607_gb300 import capi, synth

pytestmark = pytest.mark.gpu

P = 8192


@pytest.fixture(scope="module")
def torch():
    import paper_2401_01607_gb300 as pkg
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()
    capi.load()
    return t


def test_multi_full_size(torch):
    w = synth.multi(C=bench.C_STREAMS, N=bench.N_SAMPLES, L=bench.L_TAPS, block=bench.BLOCK,
                    swap_every=bench.SWAP)
    r = bench.Runner(P, w, torch)
    try:
        r.step_device()
        torch.cuda.synchronize()
        picks = bench.main_picks(96)
        got = bench.runner_outputs(r, picks)
    finally:
        r.close()
    ref = np.array([oracle.direct_at(w.x[c], w.H[c], w.vstart, m) for c, m in picks])
    err = rel_l2(got, ref)
    print(f"multi: {len(picks)} sampled outputs, rel_l2={err:.3g}")
    assert err <= TOL["fp32"]


@pytest.fixture(scope="module")
def shared_workload():
    return synth.shared(C=1024, N=240_000, L=96_000, block=256)


@pytest.mark.parametrize("prec", ["bf16split", "bf16", "fp32"])
def test_shared_full_size(torch, shared_workload, prec):
    w = shared_workload
    C, N, L, B = w.x.shape[0], w.x.shape[1], w.L, w.block
    run = bench.PushRun(torch, w.x, P, C, L)
    h_d = torch.from_numpy(np.ascontiguousarray(w.H[0][None])).cuda()
    code = {"fp32": capi.TC_FP32, "bf16": capi.TC_BF16, "bf16split": capi.TC_BF16_SPLIT}[prec]
    s = capi.tc_open_group(C, L, B, True, code, P)
    try:
        capi.tc_set_cuda_stream(s, run.ts)
        run.run(capi, s, int(h_d.data_ptr()))
        run.ts.synchronize()
        info = capi.tc_get_info(s)
        rng = np.random.default_rng(70)
        picks = [(int(rng.integers(C)), int(rng.integers(N + L - 1))) for _ in range(64)]
        got = run.outputs(picks)
    finally:
        capi.tc_close(s)
        run.close()
    if prec != "fp32":
        assert info.tensor_launches > 0 and info.fp32_fallbacks == 0
    ref = np.array([oracle.direct_at(w.x[c], w.H, w.vstart, m) for c, m in picks])
    err = rel_l2(got, ref)
    print(f"shared {prec}: {len(picks)} sampled outputs, rel_l2={err:.3g}")
    assert err <= TOL[prec]


@pytest.fixture(scope="module")
def mimo_workload():
    w = synth.mimo(N=2_880_000, L=192_000)
    nin, nout = w.mimo
    rng = np.random.default_rng(90)
    picks = [(int(rng.integers(nout)), int(rng.integers(w.x.shape[1] + w.L - 1))) for _ in range(64)]
    refs = np.array([sum(oracle.direct_at(w.x[i], w.H[0, o, i][None], w.vstart, m) for i in range(nin))
                     for o, m in picks])
    return w, picks, refs


@pytest.mark.parametrize("prec", ["bf16split", "bf16", "fp32"])
def test_mimo_full_size(torch, mimo_workload, prec):
    w, picks, refs = mimo_workload
    nin, nout = w.mimo
    L, B = w.L, w.block
    run = bench.PushRun(torch, w.x, P, nout, L)
    h_d = torch.from_numpy(np.ascontiguousarray(w.H[0])).cuda()
    code = {"fp32": capi.TC_FP32, "bf16": capi.TC_BF16, "bf16split": capi.TC_BF16_SPLIT}[prec]
    s = capi.tc_open_mimo(nin, nout, L, B, code, P)
    try:
        capi.tc_set_cuda_stream(s, run.ts)
        run.run(capi, s, int(h_d.data_ptr()))
        run.ts.synchronize()
        info = capi.tc_get_info(s)
        got = run.outputs(picks)
    finally:
        capi.tc_close(s)
        run.close()
    if prec != "fp32":
        assert info.tensor_launches > 0 and info.fp32_fallbacks == 0
    err = rel_l2(got, refs)
    print(f"mimo {prec}: {len(picks)} sampled outputs, rel_l2={err:.3g}")
    assert err <= TOL[prec]
