"""A transform held in parts: the forward and inverse TFT sharded over ranks.

The library's transforms of length n = a R + b are the row/column form of
Algorithms 1 and 2 (Section 1.3 credits this split to the cache-friendly
TFT): column q (entries x_{q + tR}) is a TFT of its own, full row rho < a is
block rho of the length-2^k network, and the ragged last row needs
E_q = C_q(omega_a) of the short columns.  The columns are independent of one
another, and so are the rows, so a transform shards as the classic
distributed four-step FFT: each of P ranks transforms a block of R / P
columns, one all-to-all exchange turns column blocks into runs of rows, each
rank transforms its rows, and the last rank assembles and transforms the
ragged row.  The inverse runs the same steps backwards, with two small
gather / scatter steps around the last row (Algorithm 2's dependency: the
long columns' row-a entries come from the last row's inverse, which needs
the short columns' E_q).

``Layout`` fixes who holds what (the same partition as include/tft.h's
tft_shard_* calls):
  * part p: column block p, columns [p W, (p + 1) W) with W = R / P, as an
    (a + 1) x W array; its long columns are j < long_cols(p);
  * part p: full rows [rho_p, rho_{p+1}), rho_p = p a // P, R words each;
  * the last part: the ragged row (b outputs) too.

The steps are plain functions of one part's data (``fwd_columns``,
``fwd_rows`` ...) with the exchanges between them done by a communicator:
``DistComm`` (torch.distributed point-to-point sends, one rank per GPU; gloo
or NCCL) or ``LocalComm`` (all parts in one process, exchanges as copies,
for a single device).  The device work goes through an ``ops`` object whose
``GpuOps`` implementation calls the CUDA library; nothing here computes a
transform value itself.
"""

import torch


class Layout:
    """Partition of a transform of length n over `parts` parts for a plan
    with row length 2^lr and n = a 2^lr + b."""

    def __init__(self, n, lr, a, b, parts):
        R = 1 << lr
        if parts < 1 or parts & (parts - 1) or parts > R:
            raise ValueError("parts must be a power of two <= R")
        self.n, self.lr, self.R, self.a, self.b = n, lr, R, a, b
        self.parts = parts
        self.W = R // parts

    @classmethod
    def for_plan(cls, plan, n, parts):
        if plan["small"] or plan["lr"] < 8:
            raise ValueError("the length's plan has no row/column split")
        return cls(n, plan["lr"], plan["a"], plan["b"], parts)

    def long_cols(self, p):
        return min(max(self.b - p * self.W, 0), self.W)

    def rows_of(self, p):
        return (p * self.a // self.parts, (p + 1) * self.a // self.parts)

    @property
    def last(self):
        return self.parts - 1

    # host-side views between one full vector and the parts (callers that
    # start from, or want, a single buffer; tests)
    def block_of(self, x, p):
        """Column block p of the length-n vector x (torch, any device)."""
        a, W, R = self.a, self.W, self.R
        blk = torch.zeros((a + 1, W), dtype=x.dtype, device=x.device)
        if a:
            blk[:a] = x[:a * R].view(a, R)[:, p * W:(p + 1) * W]
        lc = self.long_cols(p)
        if lc:
            blk[a, :lc] = x[a * R + p * W:a * R + p * W + lc]
        return blk

    def vector_of_blocks(self, blocks):
        """Inverse of block_of over all parts."""
        a, W, R = self.a, self.W, self.R
        x = torch.empty(self.n, dtype=blocks[0].dtype,
                        device=blocks[0].device)
        if a:
            x[:a * R].view(a, R).copy_(torch.cat([b[:a] for b in blocks], 1))
        for p, blk in enumerate(blocks):
            lc = self.long_cols(p)
            if lc:
                x[a * R + p * W:a * R + p * W + lc] = blk[a, :lc]
        return x

    def rows_piece(self, X, p):
        r0, r1 = self.rows_of(p)
        return X[r0 * self.R:r1 * self.R].view(r1 - r0, self.R).clone()

    def last_piece(self, X):
        return X[self.a * self.R:self.n].clone()

    def vector_of_rows(self, rows, last):
        X = torch.empty(self.n, dtype=rows[0].dtype, device=rows[0].device)
        for p, rw in enumerate(rows):
            r0, r1 = self.rows_of(p)
            X[r0 * self.R:r1 * self.R] = rw.reshape(-1)
        if self.b:
            X[self.a * self.R:] = last
        return X


class GpuOps:
    """The steps on the GPU through the library's C ABI (one context per
    device; every tensor on that device)."""

    def __init__(self, ctx, layout):
        from . import tft
        self.tft, self.ctx, self.L = tft, ctx, layout

    def columns(self, inverse, which, block, p, E):
        self.tft.tft_shard_columns(self.ctx, inverse, which, block, self.L.n,
                                   self.L.parts, p, E)

    def rows(self, inverse, rows, rho_begin):
        self.tft.tft_shard_rows(self.ctx, inverse, rows, self.L.n, rho_begin,
                                rows.shape[0])

    def last_row(self, inverse, row, E):
        self.tft.tft_shard_last_row(self.ctx, inverse, row, E, self.L.n)


# ---------------------------------------------------------------------------
# The steps of one part
# ---------------------------------------------------------------------------

def fwd_columns(L, ops, p, block):
    """Column TFTs of block p in place; returns (per-destination row
    slices, the block's share of the ragged row: long entries of row a for
    j < long_cols, E_q for the short columns)."""
    E = torch.zeros(L.W, dtype=block.dtype, device=block.device)
    ops.columns(0, 0, block, p, E)
    sends = []
    for s in range(L.parts):
        r0, r1 = L.rows_of(s)
        sends.append(block[r0:r1].contiguous())
    lc = L.long_cols(p)
    piece = E.clone()
    if lc:
        piece[:lc] = block[L.a, :lc]
    return sends, piece


def fwd_rows(L, ops, p, recvs):
    """Rows of part p from the column slices of every part, transformed."""
    rows = torch.cat(recvs, dim=1).contiguous()
    ops.rows(0, rows, L.rows_of(p)[0])
    return rows


def fwd_last(L, ops, pieces):
    """The ragged row (last part) from every part's piece: b outputs."""
    row = torch.cat(pieces).contiguous()
    E = row.clone()
    ops.last_row(0, row, E)
    return row[:L.b].clone()


def inv_rows(L, ops, p, rows):
    """Inverse rows of part p in place; returns per-destination column
    slices."""
    ops.rows(1, rows, L.rows_of(p)[0])
    return [rows[:, s * L.W:(s + 1) * L.W].contiguous()
            for s in range(L.parts)]


def inv_short_columns(L, ops, p, recvs):
    """Block p from every part's row slices; inverse of its short columns;
    returns (block, E_p)."""
    dev, dt = recvs[0].device, recvs[0].dtype
    block = torch.zeros((L.a + 1, L.W), dtype=dt, device=dev)
    for s, piece in enumerate(recvs):
        r0, r1 = L.rows_of(s)
        block[r0:r1] = piece
    E = torch.zeros(L.W, dtype=dt, device=dev)
    ops.columns(1, 0, block, p, E)
    return block, E


def inv_last(L, ops, last_out, Es):
    """Last part: the ragged row's inverse from its b outputs and every
    part's E; returns per-part pieces (the long columns' row-a entries)."""
    dev, dt = Es[0].device, Es[0].dtype
    E = torch.cat(Es).contiguous()
    row = torch.zeros(L.R, dtype=dt, device=dev)
    row[:L.b] = last_out
    ops.last_row(1, row, E)
    return [row[s * L.W:(s + 1) * L.W].clone() for s in range(L.parts)]


def inv_long_columns(L, ops, p, block, piece):
    lc = L.long_cols(p)
    if lc:
        block[L.a, :lc] = piece[:lc]
        ops.columns(1, 1, block, p, None)
    return block


# ---------------------------------------------------------------------------
# Drivers
# ---------------------------------------------------------------------------

class DistComm:
    """Exchanges between ranks by torch.distributed point-to-point sends
    (the process group's backend: NCCL on GPUs, gloo on CPUs).  Rank =
    part."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def alltoall(self, sends, recv_shapes):
        d = self.dist
        recvs = [None] * self.world
        ops = []
        for s in range(self.world):
            if s == self.rank:
                recvs[s] = sends[s].clone()
                continue
            recvs[s] = torch.empty(recv_shapes[s], dtype=sends[s].dtype,
                                   device=sends[s].device)
            ops.append(d.P2POp(d.isend, sends[s], s, self.group))
            ops.append(d.P2POp(d.irecv, recvs[s], s, self.group))
        if ops:
            for w in d.batch_isend_irecv(ops):
                w.wait()
        return recvs

    def gather_to_last(self, t):
        d, last = self.dist, self.world - 1
        if self.rank != last:
            d.send(t.contiguous(), last, self.group)
            return None
        out = []
        for s in range(self.world):
            if s == last:
                out.append(t.clone())
            else:
                buf = torch.empty_like(t)
                d.recv(buf, s, self.group)
                out.append(buf)
        return out

    def scatter_from_last(self, pieces, like):
        d, last = self.dist, self.world - 1
        if self.rank == last:
            for s in range(self.world):
                if s != last:
                    d.send(pieces[s].contiguous(), s, self.group)
            return pieces[last]
        buf = torch.empty_like(like)
        d.recv(buf, last, self.group)
        return buf


def forward_rank(L, ops, comm, block):
    """Forward TFT, run by every rank on its column block; returns (its
    rows of the transform, the ragged row's b outputs on the last rank or
    None)."""
    p = comm.rank
    sends, piece = fwd_columns(L, ops, p, block)
    r0, r1 = L.rows_of(p)
    recvs = comm.alltoall(sends, [(r1 - r0, L.W)] * L.parts)
    pieces = comm.gather_to_last(piece) if L.b else None
    rows = fwd_rows(L, ops, p, recvs)
    last = fwd_last(L, ops, pieces) if (L.b and p == L.last) else None
    return rows, last


def inverse_rank(L, ops, comm, rows, last_out=None):
    """Inverse TFT, run by every rank on its rows (the last rank also on the
    ragged row's b values); returns its column block of coefficients."""
    p = comm.rank
    sends = inv_rows(L, ops, p, rows)
    shapes = []
    for s in range(L.parts):
        r0, r1 = L.rows_of(s)
        shapes.append((r1 - r0, L.W))
    recvs = comm.alltoall(sends, shapes)
    block, E = inv_short_columns(L, ops, p, recvs)
    if L.b:
        Es = comm.gather_to_last(E)
        pieces = inv_last(L, ops, last_out, Es) if p == L.last else None
        piece = comm.scatter_from_last(pieces, E)
        block = inv_long_columns(L, ops, p, block, piece)
    return block


def forward_local(L, ops, blocks):
    """Forward TFT with every part in this process (exchanges as copies)."""
    out = [fwd_columns(L, ops, p, blocks[p]) for p in range(L.parts)]
    rows = [fwd_rows(L, ops, p, [out[s][0][p] for s in range(L.parts)])
            for p in range(L.parts)]
    last = fwd_last(L, ops, [o[1] for o in out]) if L.b else None
    return rows, last


def inverse_local(L, ops, rows, last_out=None):
    sends = [inv_rows(L, ops, p, rows[p]) for p in range(L.parts)]
    got = [inv_short_columns(L, ops, p, [sends[s][p]
                                         for s in range(L.parts)])
           for p in range(L.parts)]
    blocks = [g[0] for g in got]
    if L.b:
        pieces = inv_last(L, ops, last_out, [g[1] for g in got])
        blocks = [inv_long_columns(L, ops, p, blocks[p], pieces[p])
                  for p in range(L.parts)]
    return blocks
