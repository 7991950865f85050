"""Sharding one array over several devices (host-side logic).

Every block of the APAX encoder is coded on its own (Sec. 6); only the
best-stream decision of a block reads the block before it.  An array of nb
blocks is therefore split into contiguous block ranges, one per rank; rank r
encodes its range with the halo block before it (apax_encode_shard) into a
container of its own sub-array.  Fixed rate needs no exchange: packet j sits
at j*B.  Fixed quality has one exchange step: an all-gather of one payload
size per rank, whose exclusive scan gives each rank's word offset in the
whole payload; apax_shard_rebase adds it to the rank's offset-table slice.
The shards then stay distributed or are gathered and merged
(apax_merge_shards on one device, or `merge_host` on host bytes) into the
container a single call would have written.

Only the block arithmetic below and torch.distributed's collective run on
the host; every sample is coded by the library's kernels.
"""
from __future__ import annotations

import struct


def block_ranges(nb: int, world: int):
    """Contiguous block ranges [b0, b1) of nb blocks over `world` ranks
    (sizes differ by at most one; a rank may get none when nb < world)."""
    return [(nb * r // world, nb * (r + 1) // world) for r in range(world)]


def halo_elements(n: int, block_size: int, b0: int, b1: int):
    """Element range [e0, e1) a rank must hold to encode blocks [b0, b1):
    its own elements and the whole block before them."""
    e0 = (b0 - 1) * block_size if b0 > 0 else 0
    return e0, min(b1 * block_size, n)


def table_bytes(blocks: int) -> int:
    return (4 * blocks + 7) // 8 * 8


def payload_bytes(container_bytes: int, blocks: int, fixed_quality: bool) -> int:
    """Payload bytes of a shard container (header and offset table off)."""
    return container_bytes - 40 - (table_bytes(blocks) if fixed_quality else 0)


def exclusive_offsets(sizes):
    """Exclusive prefix sums (the payload offset of every shard)."""
    out, acc = [], 0
    for v in sizes:
        out.append(acc)
        acc += v
    return out, acc


def exchange_payload_sizes(my_payload: int, group=None):
    """The exchange step of a fixed-quality shard: all-gather one payload
    size per rank (torch.distributed), then this rank's byte offset in the
    whole payload and the total."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else "cpu"
    mine = torch.tensor([my_payload], dtype=torch.int64, device=dev)
    allv = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(allv, mine, group=group)
    sizes = [int(t.item()) for t in allv]
    offs, total = exclusive_offsets(sizes)
    return offs[dist.get_rank(group)], total, sizes


def merge_host(shards, ranges, n: int, fixed_quality: bool) -> bytes:
    """The whole-array container from shard containers held as host bytes
    (rank order): the first shard's header with the whole array's element
    count and payload size, the offset-table slices with each shard's word
    offset added, then the payloads."""
    nb = ranges[-1][1] if ranges else 0
    head = bytearray(shards[0][:40])
    pays, tables = [], []
    for c, (b0, b1) in zip(shards, ranges):
        nbs = b1 - b0
        h = 40 + (table_bytes(nbs) if fixed_quality else 0)
        pays.append(bytes(c[h:]))
        if fixed_quality:
            tables.append(struct.unpack_from(f"<{nbs}I", c, 40))
    offs, total = exclusive_offsets([len(p) for p in pays])
    struct.pack_into("<Q", head, 20, n)
    struct.pack_into("<Q", head, 28, total)
    table = b""
    if fixed_quality:
        words = []
        for t, o in zip(tables, offs):
            words.extend(v + o // 4 for v in t)
        if any(w > 0xFFFFFFFF for w in words):
            raise OverflowError("payload beyond 2^32 words")
        table = struct.pack(f"<{nb}I", *words)
        table += b"\0" * (table_bytes(nb) - len(table))
    return bytes(head) + table + b"".join(pays)
