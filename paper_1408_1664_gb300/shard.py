"""One job split over W = 2^k ranks, one GPU each.

The split is the paper's hypercube decomposition of the subset lattice
(Section 3.2): the top k variables of the step-3 tile index name the rank, so
every rank computes 1/W of the tiles of every popcount level of the forward
sum F (Eq. 9) and of the backward sum R' (Eq. 10), then the ranks exchange the
level before any of them computes the next (a level-hl tile reads level
hl - 1 of F, or hl + 1 of R', from the other ranks' sub-lattices).  The two
sweeps are independent, so one exchange step carries F level st and R' level
H - st together: H + 1 all-gathers in all.  Steps 1-2 (scores, A) run whole on
every rank; steps 4-5 (Gamma_v, Eq. 12, and the edge sums, Eq. 11) run on each
rank for the endpoints v with v mod W = rank, and one all-reduce of the n x n
posterior matrix ends the job.  The library (include/bnedge.h, "Shards")
computes and packs; this module moves the packed levels:

  run_virtual  all W ranks in this process on one device, each with its own
               shard, the exchange a set of device-buffer reads (the ranks'
               buffers are all on this device);
  run_rank     this process is one rank; the exchange is a
               torch.distributed all_gather_into_tensor (NCCL on GPUs), the
               end an all_reduce.

Both drive any object with the Shard interface (level, exchange_bytes, pack,
unpack, finish, levels), which is how the exchange schedule is tested on CPU
ranks.
"""
from __future__ import annotations


def steps(levels: int):
    """(F level, R' level) of each exchange step: F from the empty set up,
    R' from the full set down."""
    return [(st, levels - st) for st in range(levels + 1)]


def step_bytes(shard, hf: int, hr: int) -> tuple[int, int]:
    """Bytes of the F part and of the R' part of one rank's step buffer."""
    return shard.exchange_bytes(hf), shard.exchange_bytes(hr)


def max_step_bytes(shard) -> int:
    return max(sum(step_bytes(shard, hf, hr)) for hf, hr in steps(shard.levels))


def run_virtual(shards, bufs, post_parts, lpd, stream=None) -> None:
    """All ranks of one job in this process.  shards: one per rank, in rank
    order; bufs: one byte buffer per rank of at least max_step_bytes; post_parts:
    one n x n device buffer per rank (each gets its endpoints' columns, zeros
    elsewhere; their sum is the posterior matrix); lpd: one double (log P(D),
    written by rank 0)."""
    for sh in shards:
        sh.prepare(stream)
    for hf, hr in steps(shards[0].levels):
        bf, br = step_bytes(shards[0], hf, hr)
        for sh in shards:
            sh.level(0, hf, stream)
            sh.level(1, hr, stream)
        for sh, b in zip(shards, bufs):
            sh.pack(0, hf, b[:bf], stream)
            sh.pack(1, hr, b[bf:bf + br], stream)
        for sh in shards:
            for q, b in enumerate(bufs):
                sh.unpack(0, hf, q, b[:bf], stream)
                sh.unpack(1, hr, q, b[bf:bf + br], stream)
    for q, (sh, part) in enumerate(zip(shards, post_parts)):
        sh.finish(part, lpd if q == 0 else None, stream)


def run_rank(shard, dist, buf, gathered, post, lpd=None, stream=None, group=None) -> None:
    """This process's rank of one job.  buf: max_step_bytes bytes; gathered:
    W times that, on the collective's device; post: n x n doubles, the whole
    posterior matrix on return (every rank); lpd: one double or None.  The
    collectives order themselves against the current torch stream, which
    `stream` must be (or None with the library on its context's stream
    synchronised by the caller)."""
    W = shard.world
    shard.prepare(stream)
    for hf, hr in steps(shard.levels):
        bf, br = step_bytes(shard, hf, hr)
        nb = bf + br
        shard.level(0, hf, stream)
        shard.level(1, hr, stream)
        shard.pack(0, hf, buf[:bf], stream)
        shard.pack(1, hr, buf[bf:nb], stream)
        dist.all_gather_into_tensor(gathered[:W * nb], buf[:nb], group=group)
        for q in range(W):
            o = q * nb
            shard.unpack(0, hf, q, gathered[o:o + bf], stream)
            shard.unpack(1, hr, q, gathered[o + bf:o + nb], stream)
    shard.finish(post, lpd, stream)
    dist.all_reduce(post, op=dist.ReduceOp.SUM, group=group)
