"""Helpers shared by the GPU parity tests: drive the C ABI and compare with the oracle."""
from __future__ import annotations

import numpy as np

from paper_2401_01607_gb300 import capi

# Tolerances on relative L2 error against the FP64 oracle, by precision.
TOL = {"fp32": 1e-6, "bf16split": 1e-5, "bf16": 3e-3}


def rel_l2(y, ref):
    y = np.asarray(y, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.linalg.norm(y - ref) / max(np.linalg.norm(ref), 1e-300))


def max_abs(y, ref):
    return float(np.max(np.abs(np.asarray(y, np.float64) - np.asarray(ref, np.float64))))


def stream_host(x, H, vstart, L, block, pushes=None, max_push=0, shared_ir=True, ramps=None, precision=None):
    """Streams x ([C, N] or [N]) through a group via host-pointer pushes and
    returns [C, N + L - 1] float32 (input then flush tail).
    H: [nver, L'] shared, or [C, nver, L'] per channel. vstart: [nver].
    ramps: crossfade length of each switch ([nver], entry 0 unused)."""
    x = np.atleast_2d(np.asarray(x, np.float32))
    C, N = x.shape
    H = np.asarray(H, np.float32)
    per_channel = H.ndim == 3
    mp = max_push or block
    if C == 1 and not per_channel and mp == block and precision is None:
        s = capi.tc_open_stream(L, block)
    else:
        s = capi.tc_open_group(C, L, block, not per_channel, capi.TC_FP32 if precision is None else precision, mp)
    try:
        if len(vstart) > 4:
            capi.tc_set_max_versions(s, min(16, len(vstart) + 1))
        outs = []
        pos = 0
        v_next = 0
        sizes = pushes or []
        i = 0
        while pos < N:
            n = sizes[i] if i < len(sizes) else mp
            i += 1
            n = min(n, N - pos)
            # Register every version that starts before the end of this push.
            while v_next < len(vstart) and vstart[v_next] < pos + n:
                if ramps is not None:
                    capi.tc_set_crossfade(s, int(ramps[v_next]) if v_next > 0 else 1)
                rows = H[:, v_next] if per_channel else H[v_next][None]
                capi.tc_set_ir_rows(s, np.ascontiguousarray(rows), rows.shape[-1], max(int(vstart[v_next]), pos))
                v_next += 1
            y = np.empty((C, n), np.float32)
            capi.tc_push(s, np.ascontiguousarray(x[:, pos:pos + n]), n, y)
            outs.append(y)
            pos += n
        tail = np.empty((C, L - 1), np.float32)
        if L > 1:
            capi.tc_flush(s, tail, L - 1)
        outs.append(tail)
    finally:
        capi.tc_close(s)
    return np.concatenate(outs, axis=1)
