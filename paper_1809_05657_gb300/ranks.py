"""Logical devices on several ranks (one process per GPU): the transport of cross-rank sections.

The paper runs one MPI process per device; every process keeps every process's section sets
(Sec. 2.1), so all processes compute the same messages, and messages travel by MPI
(Sec. 3.1, HDArrayApplyKernel).  Here every rank runs the same HDArray program on the same
logical devices; HDArraySetRankMap tells the library which devices are this rank's, so it keeps
buffers and runs kernels for those only.  The replicated bookkeeping gives every rank the same
cross-rank records for each call (HDArrayGetRankPlan), in the same order, without any exchange of
metadata.  For each (source rank, destination rank) pair, all records of one array in one call
travel as one message:

  * the source rank packs the records' boxes into a staging buffer with the library's copy kernel
    (HDArrayPackBoxes; layout: each box row-major, 16-byte aligned, records in order);
  * the buffers cross with torch.distributed point-to-point operations, NCCL between GPUs and
    gloo between CPU processes (send and receive posted together, so no rank waits on a send
    before posting its receives);
  * the destination rank unpacks them into its devices' buffers (HDArrayUnpackBoxes).

The library calls the transport after a call's bookkeeping and before its kernel, so the kernel
reads the received sections.  Sections between two devices of one rank stay device copies inside
the library (fused into the stencil launches).  No collective other than these point-to-point
messages is used, and no rank reads another rank's memory.
"""
import numpy as np

from . import hdarray as H

RECORD = H.HDARRAY_RANK_RECORD


def staging_layout(esize, records):
    """Byte offset of each record's box in a staging buffer and the total size: each box row-major,
    starting at the first 16-byte boundary after the previous one (the library's layout)."""
    offs, total = [], 0
    for r in records:
        total = (total + 15) // 16 * 16
        offs.append(total)
        total += int(np.prod(np.asarray(r[7:10]) - np.asarray(r[4:7]))) * esize
    return offs, total


class RankTransport:
    """The transport callback (HDArraySetTransport) for one rank.

    pack(array, records, staging, nbytes) and unpack(array, records, staging, nbytes) move the
    records' boxes between this rank's device buffers and a staging tensor; by default they are
    the library's HDArrayPackBoxes / HDArrayUnpackBoxes on staging tensors in GPU memory.  A test
    on CPU processes passes host-side ones and device="cpu" (gloo)."""

    def __init__(self, rank, device="cuda", pack=None, unpack=None, group=None):
        self.rank = rank
        self.device = device
        self.pack = pack or self._lib_pack
        self.unpack = unpack or self._lib_unpack
        self.group = group
        self.messages = 0
        self.bytes_sent = 0

    @staticmethod
    def _lib_pack(array, recs, staging, nbytes):
        H.HDArrayPackBoxes(array, recs, staging, nbytes)  # synchronous on the library stream

    @staticmethod
    def _lib_unpack(array, recs, staging, nbytes):
        H.HDArrayUnpackBoxes(array, recs, staging, nbytes)

    def _nbytes(self, array, recs):
        return H.HDArrayStagingBytes(array, recs)

    def __call__(self, array, recs, stream):
        import torch
        import torch.distributed as dist
        me = self.rank
        sends, recvs = {}, {}
        for i, r in enumerate(recs):
            if int(r[2]) == me:
                sends.setdefault(int(r[3]), []).append(i)
            elif int(r[3]) == me:
                recvs.setdefault(int(r[2]), []).append(i)
        ops, inbound = [], []
        for peer in sorted(sends):
            sub = recs[sends[peer]]
            n = self._nbytes(array, sub)
            buf = torch.empty(n, dtype=torch.uint8, device=self.device)
            self.pack(array, sub, buf, n)
            ops.append(dist.P2POp(dist.isend, buf, peer, self.group))
            self.messages += 1
            self.bytes_sent += n
        for peer in sorted(recvs):
            sub = recs[recvs[peer]]
            n = self._nbytes(array, sub)
            buf = torch.empty(n, dtype=torch.uint8, device=self.device)
            ops.append(dist.P2POp(dist.irecv, buf, peer, self.group))
            inbound.append((sub, buf, n))
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()
            if self.device != "cpu":
                torch.cuda.synchronize()  # the received bytes are in place before the unpack reads them
        for sub, buf, n in inbound:
            self.unpack(array, sub, buf, n)
        return 0


def allreduce_partial(value, op):
    """Combine the per-rank partial results of HDArrayReduce (each rank folds its own devices):
    SUM, PROD, MAX or MIN over the ranks."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    dop = {H.SUM: dist.ReduceOp.SUM, H.PROD: dist.ReduceOp.PRODUCT, H.MAX: dist.ReduceOp.MAX,
           H.MIN: dist.ReduceOp.MIN}[op]
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dop)
    return float(t.item())
