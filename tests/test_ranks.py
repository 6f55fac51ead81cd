"""Logical devices on two ranks (gloo, CPU processes): the cross-rank exchange.

Each rank runs the same Jacobi program with the same logical devices, the library in host-only
mode (bookkeeping without buffers) and a rank map that gives each rank half of the devices.  The
devices' buffers are numpy arrays held by the rank that owns the device; the transport
(paper_1809_05657_gb300.ranks.RankTransport) moves every cross-rank section through gloo, with
host-side pack/unpack in the library's staging layout; the rank itself copies the sections
between its own devices and runs the Jacobi step on its devices' work boxes.  After every call:

  * the exchange equals the oracle's messages element by element, and the cross-rank records are
    exactly its moves between devices of different ranks, the same list on both ranks;
  * every element each device holds (the oracle's per-device flags) equals the global value bit
    for bit -- so everything that crossed ranks landed where it belongs.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.environ["ROOT"])
sys.path.insert(0, os.path.join(os.environ["ROOT"], "tests"))
import numpy as np
import torch.distributed as dist
import oracle
import synthetic
from harness import rasterise
from paper_1809_05657_gb300 import hdarray as H
from paper_1809_05657_gb300.ranks import RankTransport, staging_layout

rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
case = json.loads(os.environ["CASE"])
dims, P, ptype, rmap, iters, dtype = (tuple(case["dims"]), case["P"], case["ptype"], case["rmap"],
                                      case["iters"], case["dtype"])
np_t = {"double": np.float64, "float": np.float32}[dtype]
dist.init_process_group("gloo")
local = [p for p in range(P) if rmap[p] == rank]

# host stand-ins for this rank's device buffers: buf[array][device] covers the whole index space
buf = {n: {p: np.zeros(dims, np_t) for p in local} for n in ("B", "A")}

def box_of(r):
    return tuple(slice(int(r[4 + d]), int(r[7 + d])) for d in range(len(dims)))

def pack(array, recs, staging, nbytes):
    offs, total = staging_layout(np.dtype(np_t).itemsize, recs)
    assert total == nbytes
    st = staging.numpy()
    for r, off in zip(recs, offs):
        assert rmap[int(r[0])] == rank
        blk = np.ascontiguousarray(buf[array.sym][int(r[0])][box_of(r)])
        st[off: off + blk.nbytes] = blk.view(np.uint8).ravel()

def unpack(array, recs, staging, nbytes):
    offs, total = staging_layout(np.dtype(np_t).itemsize, recs)
    assert total == nbytes
    st = staging.numpy()
    for r, off in zip(recs, offs):
        assert rmap[int(r[1])] == rank
        dst = buf[array.sym][int(r[1])][box_of(r)]
        dst[...] = st[off: off + dst.size * dst.itemsize].view(np_t).reshape(dst.shape)

tr = RankTransport(rank, device="cpu", pack=pack, unpack=unpack)
H.HDArrayInit(ndev=P, host_only=True)
H.HDArraySetRankMap(rmap, rank)
H.HDArraySetTransport(tr)
B = H.HDArrayCreate("B", dtype, None, *dims)
A = H.HDArrayCreate("A", dtype, None, *dims)
D = H.HDArrayPartition(ptype, dims, (0, 0), dims, P)
W = H.HDArrayPartition(ptype, dims, (1, 1), (dims[0] - 1, dims[1] - 1), P)
x = synthetic.jacobi_field(dims, stream=41, dtype=dtype)

o = oracle.Oracle(P)
OB, OA = o.create("B", dtype, dims), o.create("A", dtype, dims)
od = o.partition(ptype, dims, (0, 0), dims)
ow = o.partition(ptype, dims, (1, 1), (dims[0] - 1, dims[1] - 1))
lib_of = {"B": B, "A": A}
orc_of = {"B": OB, "A": OA}

H.HDArrayWrite(B, x, D)   # bookkeeping; the data goes into this rank's devices' regions
o.write(OB, x, od)
for p in local:
    lo, hi = o.parts[od][p]
    buf["B"][p][lo[0]:hi[0], lo[1]:hi[1]] = x[lo[0]:hi[0], lo[1]:hi[1]]

def check_exchange(name, msgs):
    moves = H.HDArrayGetPlan(lib_of[name])
    got = rasterise(moves, dims, P)
    assert np.array_equal(got, msgs.src.astype(np.int32)), "exchange differs from the oracle"
    recs = H.HDArrayGetRankPlan(lib_of[name])
    cross = sorted((s, d, lo[:2], hi[:2]) for s, d, lo, hi in moves if rmap[s] != rmap[d])
    mine = sorted((int(r[0]), int(r[1]), tuple(int(v) for v in r[4:6]), tuple(int(v) for v in r[7:9])) for r in recs)
    assert mine == [(s, d, tuple(lo), tuple(hi)) for s, d, lo, hi in cross]
    assert all(int(r[2]) == rmap[int(r[0])] and int(r[3]) == rmap[int(r[1])] for r in recs)
    lists = [None] * world
    dist.all_gather_object(lists, recs.tolist())
    assert all(l == lists[0] for l in lists), "ranks disagree on the cross-rank records"
    for s, d, lo, hi in moves:  # sections between two of this rank's devices: a local copy
        if rmap[s] == rank and rmap[d] == rank:
            sl = (slice(lo[0], hi[0]), slice(lo[1], hi[1]))
            buf[name][d][sl] = buf[name][s][sl]
    return len(recs)

def check_held():
    for name in ("B", "A"):
        owner, have = orc_of[name].state_get()
        G = orc_of[name].G.reshape(-1)
        for p in local:
            held = have[p].astype(bool) & (owner >= 0)
            got = buf[name][p].reshape(-1)[held]
            assert np.array_equal(got.view(np.uint8), G[held].view(np.uint8)), "device %d of %s" % (p, name)

ncross = 0
X, Y = "B", "A"
for it in range(iters):
    H.HDArrayApplyKernel("jacobi2d", W, lib_of[X], lib_of[Y])   # the transport runs inside
    msgs = o.apply("jacobi2d", ow, [orc_of[X], orc_of[Y]])
    ncross += check_exchange(X, msgs[0])
    for p in local:          # the step on this rank's devices, each reading only its own buffer
        lo, hi = o.parts[ow][p]
        s, t = buf[X][p], buf[Y][p]
        r0, r1, c0, c1 = lo[0], hi[0], lo[1], hi[1]
        v = s[r0:r1, c0 - 1:c1 - 1] + s[r0:r1, c0 + 1:c1 + 1]
        v = v + s[r0 - 1:r1 - 1, c0:c1]
        v = v + s[r0 + 1:r1 + 1, c0:c1]
        t[r0:r1, c0:c1] = v * np_t(0.25)
    check_held()
    X, Y = Y, X

# Read by the data partition: ownership moves back to the data devices, across ranks too
out = np.zeros(dims, np_t)
H.HDArrayRead(lib_of[X], out, D)
msgs = o.read(orc_of[X], od)
ncross += check_exchange(X, msgs)
check_held()
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "cross_records": ncross, "messages": tr.messages, "bytes": tr.bytes_sent}))
"""

CASES = [
    {"dims": [40, 36], "P": 4, "ptype": 2, "rmap": [0, 0, 1, 1], "iters": 4, "dtype": "double"},  # BLOCK 2x2
    {"dims": [33, 50], "P": 4, "ptype": 1, "rmap": [0, 1, 0, 1], "iters": 5, "dtype": "float"},   # COL
    {"dims": [45, 29], "P": 3, "ptype": 0, "rmap": [1, 0, 1], "iters": 3, "dtype": "float"},      # ROW
]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("case", CASES, ids=["block2x2", "col_alternating", "row3"])
def test_cross_rank_exchange_two_gloo_ranks(case):
    pytest.importorskip("torch.distributed")
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), ROOT=ROOT, CUDA_VISIBLE_DEVICES="", CASE=json.dumps(case))
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-3000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert outs[0]["cross_records"] == outs[1]["cross_records"] > 0
    assert outs[0]["messages"] > 0 and outs[1]["messages"] > 0   # both ranks sent sections


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["float", "double", "bf16"])
def test_pack_unpack_boxes_gpu(dtype):
    """HDArrayPackBoxes / HDArrayUnpackBoxes on one GPU: the boxes of a call's exchange packed from
    their source devices' buffers into a staging buffer in GPU memory equal the oracle's values in
    the staging layout, bit for bit; a pattern unpacked into the destination devices' buffers reads
    back unchanged."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import numpy as np
    import oracle
    import synthetic
    from __graft_entry__ import build_library
    from paper_1809_05657_gb300 import hdarray as H
    from paper_1809_05657_gb300.ranks import staging_layout
    build_library()
    dims, P = (70, 93), 4
    np_t = {"double": np.float64, "float": np.float32, "bf16": np.uint16}[dtype]
    x = synthetic.jacobi_field(dims, stream=42, dtype=dtype)
    H.HDArrayInit(ndev=P)
    try:
        B = H.HDArrayCreate("B", dtype, None, *dims)
        A = H.HDArrayCreate("A", dtype, None, *dims)
        D = H.HDArrayPartition(H.BLOCK, dims, (0, 0), dims, P)
        W = H.HDArrayPartition(H.BLOCK, dims, (1, 1), (dims[0] - 1, dims[1] - 1), P)
        H.HDArrayWrite(B, x, D)
        H.HDArrayApplyKernel("jacobi2d", W, B, A)
        H.HDArrayApplyKernel("jacobi2d", W, A, B)
        moves = H.HDArrayGetPlan(A)  # A's exchange of the second call (every device received)
        assert moves
        recs = np.array([[s, d, 0, 0, lo[0], lo[1], lo[2], hi[0], hi[1], hi[2]] for s, d, lo, hi in moves],
                        np.int64)
        n = H.HDArrayStagingBytes(A, recs)
        offs, total = staging_layout(np.dtype(np_t).itemsize, recs)
        assert n == total
        stg = torch.zeros(n, dtype=torch.uint8, device="cuda")
        H.HDArrayPackBoxes(A, recs, stg, n)
        got = stg.cpu().numpy()
        o = oracle.Oracle(P)
        ob, oa = o.create("B", dtype, dims), o.create("A", dtype, dims)
        o.write(ob, x, o.partition(oracle.BLOCK, dims, (0, 0), dims))
        o.apply("jacobi2d", o.partition(oracle.BLOCK, dims, (1, 1), (dims[0] - 1, dims[1] - 1)), [ob, oa])
        for r, off in zip(recs, offs):
            want = np.ascontiguousarray(oa.G[r[4]:r[7], r[5]:r[8]])
            assert np.array_equal(got[off: off + want.nbytes], want.view(np.uint8).ravel())
        pattern = (np.arange(n) % 251).astype(np.uint8)
        H.HDArrayUnpackBoxes(A, recs, torch.from_numpy(pattern).cuda(), n)
        for r, off in zip(recs, offs):
            shape = (int(r[7] - r[4]), int(r[8] - r[5]))
            back = np.zeros(shape, np_t)
            H.HDArrayReadDeviceBuffer(A, int(r[1]), (int(r[4]), int(r[5])), (int(r[7]), int(r[8])), back)
            assert np.array_equal(back.view(np.uint8).ravel(), pattern[off: off + back.nbytes])
        # records naming a device that is not this rank's, or a box outside the buffer, are refused
        bad = recs[:1].copy()
        bad[0, 7] = dims[0] + 1
        with pytest.raises(H.HDArrayError):
            H.HDArrayPackBoxes(A, bad, stg, n)
    finally:
        H.HDArrayExit()
