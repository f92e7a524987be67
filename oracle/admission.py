"""Block admission rule — oracle (test infrastructure).

Sec. 2.1: the block scheduler places a block on an SM only if the SM still has
enough of every per-SM resource (block slots, threads, registers, shared memory)
for the whole block; Sec. 4.2 works the register case through on an H100.
"""
from __future__ import annotations


def free_after(total: int, used_per_block: int, resident_blocks: int) -> int:
    return total - used_per_block * resident_blocks


def admits(sm: dict, resident: list, block: dict) -> bool:
    """sm: capacities {'blocks','threads','regs','smem'}; resident: list of blocks
    already on the SM, each {'threads','regs' (per block),'smem'}; block: the
    candidate.  True when every resource still has room for the candidate."""
    for key in ("threads", "regs", "smem"):
        used = sum(b[key] for b in resident)
        if used + block[key] > sm[key]:
            return False
    return len(resident) + 1 <= sm["blocks"]
