"""One page split over several GPUs by bands of rows.

Section 2's within- and between-class scatter matrices are sums over the
training pixels, so a page cut into parts gives, part by part, exact integer
class moments that add up to the whole page's.  The protocol (one process
and one GPU per part):

1. ``moments()``: the part's class moments (cva_fit_moments +
   cva_model_moments) and its device status;
2. the moments are summed over all parts (int64, exact) and the statuses
   reduced by min (errors are negative), so every part sees the page's;
3. ``fit(total)``: every part finishes the same fit from the page's moments
   (cva_fit_from_moments: bit-identical to cva_fit on the whole page) and
   forms the training-score range of its own training pixels;
4. the parts' ranges merge: min over the low ends, max over the high ends;
5. ``project(range, out)``: the part's 8-bit image with the page's range.

The only data exchanged are K (B+1)(B+2)/2 int64 words and 2 k floats.
``run_split`` drives one part through the protocol with torch.distributed
collectives; the phases are separate so that tests can also drive several
parts from one process.  Every computation is the CUDA library's; this
module only moves tensors.
"""
from __future__ import annotations

from typing import Optional, Tuple

import torch

from . import _lib as L


def row_band(H: int, parts: int, index: int) -> Tuple[int, int]:
    """Rows [r0, r1) of part `index` of `parts`: equal bands, the first
    H % parts parts one row longer."""
    if not (0 <= index < parts) or parts < 1:
        raise ValueError("bad part index")
    base, extra = divmod(H, parts)
    r0 = index * base + min(index, extra)
    return r0, r0 + base + (1 if index < extra else 0)


class PagePart:
    """One part (a band of rows) of a page on this process's GPU."""

    def __init__(self, cube: torch.Tensor, labels: torch.Tensor, K: int, k: int, stream=None,
                 max_train: Optional[int] = None):
        self.cube, self.labels, self.K, self.k = cube, labels, K, k
        self.B = int(cube.shape[0])
        self.stream = stream
        self.model = L.Model(self.B, K)
        if max_train is not None:
            L.cva_model_reserve(self.model, max_train)
        L.cva_set_variates(self.model, k)

    def moments(self) -> Tuple[torch.Tensor, int]:
        mom = torch.empty(L.moment_words(self.B, self.K), dtype=torch.int64, device=self.cube.device)
        L.cva_fit_moments(self.cube, self.labels, self.K, self.model, stream=self.stream)
        L.cva_model_moments(self.model, mom, stream=self.stream)
        return mom, L.cva_status(self.model, stream=self.stream)

    def fit(self, total: torch.Tensor) -> Tuple[torch.Tensor, int]:
        L.cva_fit_from_moments(self.model, total, stream=self.stream)
        rng = torch.empty(2 * self.k, dtype=torch.float32, device=self.cube.device)
        L.cva_model_training_range(self.model, rng, stream=self.stream)
        return rng, L.cva_status(self.model, stream=self.stream)

    def project(self, rng: torch.Tensor, out: torch.Tensor) -> None:
        L.cva_set_training_range(self.model, rng, stream=self.stream)
        L.cva_project_u8(self.cube, self.model, self.k, L.CVA_RANGE_TRAINING, out, stream=self.stream)

    def close(self) -> None:
        self.model.close()


def merge_ranges(lo: torch.Tensor, hi: torch.Tensor) -> torch.Tensor:
    """(lo_0, hi_0, lo_1, hi_1, ..) from the merged low and high ends."""
    out = torch.empty(2 * lo.numel(), dtype=lo.dtype, device=lo.device)
    out[0::2] = lo
    out[1::2] = hi
    return out


def run_split(part, out: torch.Tensor, group=None) -> None:
    """Drive `part` (a PagePart, or any object with the same three phases)
    through the protocol, exchanging with the other parts of the page over
    torch.distributed (`group`: the page's process group).  Raises
    CvaError with the page's first device error."""
    import torch.distributed as dist

    mom, st = part.moments()
    code = torch.tensor([st], dtype=torch.int64, device=mom.device)
    dist.all_reduce(code, op=dist.ReduceOp.MIN, group=group)
    if int(code.item()) != L.CVA_OK:
        raise L.CvaError(int(code.item()), "split fit (moments)")
    dist.all_reduce(mom, op=dist.ReduceOp.SUM, group=group)
    rng, st = part.fit(mom)
    code = torch.tensor([st], dtype=torch.int64, device=mom.device)
    dist.all_reduce(code, op=dist.ReduceOp.MIN, group=group)
    if int(code.item()) != L.CVA_OK:
        raise L.CvaError(int(code.item()), "split fit")
    lo = rng[0::2].contiguous()
    hi = rng[1::2].contiguous()
    dist.all_reduce(lo, op=dist.ReduceOp.MIN, group=group)
    dist.all_reduce(hi, op=dist.ReduceOp.MAX, group=group)
    part.project(merge_ranges(lo, hi), out)
