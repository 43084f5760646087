"""Calls on one gauge handle from several host threads and streams.

The library's shared operator scratch (M^dag M's intermediate field, the
Schur operator's three half-volume fields) and its solver and contraction
workspaces are guarded on the host and ordered across streams on the GPU.
Two threads, each on its own stream, apply M^dag M and the Schur operator
and run solves and contractions on one handle at the same time (ctypes
releases the interpreter lock during the calls); every result equals the
same call made alone.  A further thread runs the truncated-solver driver
(which itself uses a worker thread and a second stream) while the main
thread applies operators on the same handle.
"""
import threading

import numpy as np
import pytest
import torch

from gpu_helpers import gauge
from oracle import momenta
from paper_1401_6750_gb300 import abi, api

pytestmark = pytest.mark.gpu


def _run_threads(fns):
    errs = []

    def wrap(fn):
        try:
            fn()
        except Exception as e:  # reported below
            errs.append(e)
    ts = [threading.Thread(target=wrap, args=(f,)) for f in fns]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errs, errs


def test_two_threads_share_operator_scratch(ctx):
    dims = (8, 8, 8, 16)
    g, _ = gauge(ctx, dims, 0.3, 21, -1, precs=(abi.TSM_F32,))
    prec, n, reps = abi.TSM_F32, 4, 20
    srcs = [g.sources(900 + k, 0, n, prec) for k in range(2)]
    ops = (abi.TSM_OP_MDAGM, abi.TSM_OP_MHAT)
    want = [[g.dslash(op, 0.125, 0.01, prec, srcs[k], n).clone() for op in ops] for k in range(2)]
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in range(2)]
    got = [[None, None] for _ in range(2)]

    def worker(k):
        def run():
            with torch.cuda.stream(streams[k]):
                for _ in range(reps):
                    for j, op in enumerate(ops):
                        got[k][j] = g.dslash(op, 0.125, 0.01, prec, srcs[k], n, stream=streams[k])
            streams[k].synchronize()
        return run
    _run_threads([worker(0), worker(1)])
    for k in range(2):
        for j in range(2):
            assert torch.equal(got[k][j], want[k][j]), (k, j)
    g.close()


def test_solves_and_contractions_from_two_threads(ctx):
    dims = (6, 4, 4, 8)
    g, _ = gauge(ctx, dims, 0.3, 22, -1)
    moms = momenta.momentum_list(4)
    solver = abi.TSM_SOLVER_LP_F16 | abi.TSM_SOLVER_EO

    def job(seed, stream=None):
        sol, _ = g.solve_sources(0.125, 0.01, solver, 1e-2, seed, 0, 3, stream=stream)
        return api.loops_complex(g.contract(0.125, 0.01, abi.TSM_F32, sol, 3, moms, stream=stream))
    want = [job(31), job(32)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    got = [None, None]

    def worker(k):
        def run():
            with torch.cuda.stream(streams[k]):
                for _ in range(3):
                    got[k] = job(31 + k, stream=streams[k])
        return run
    _run_threads([worker(0), worker(1)])
    for k in range(2):
        assert np.array_equal(got[k], want[k]), k
    g.close()


def test_tsm_driver_beside_operator_calls(ctx):
    dims = (6, 4, 4, 8)
    g, _ = gauge(ctx, dims, 0.3, 23, -1)
    moms = momenta.momentum_list(4)
    eo = abi.TSM_SOLVER_EO
    args = (0.125, 0.01, 8, 3, 1e-2, 1e-8, abi.TSM_SOLVER_LP_F16 | eo, abi.TSM_SOLVER_F32_RELIABLE | eo, 41, moms)
    want, _ = g.tsm(*args, nrhs_per_launch=4)
    src = g.sources(42, 0, 2, abi.TSM_F32)
    ref = g.dslash(abi.TSM_OP_MHATDAG, 0.125, 0.01, abi.TSM_F32, src, 2).clone()
    torch.cuda.synchronize()
    s_tsm, s_op = torch.cuda.Stream(), torch.cuda.Stream()
    out = {}

    def tsm_job():
        with torch.cuda.stream(s_tsm):
            out["tsm"] = g.tsm(*args, nrhs_per_launch=4, stream=s_tsm)[0]

    def op_job():
        with torch.cuda.stream(s_op):
            for _ in range(50):
                out["op"] = g.dslash(abi.TSM_OP_MHATDAG, 0.125, 0.01, abi.TSM_F32, src, 2, stream=s_op)
        s_op.synchronize()
    _run_threads([tsm_job, op_job])
    assert np.array_equal(out["tsm"], want)
    assert torch.equal(out["op"], ref)
    g.close()
