"""Batches of independent banded systems of uneven n and k, solved by one
CUDA-graph launch.

Every system gets its own graph-safe LR-SPIKE handle (factor and solve only
enqueue work: up to `iterations` FP64 refinement steps, no host reads) on one
of a pool of side streams.  The residual that meets tol raises a device flag
of its system, and the kernels of that system's remaining steps return at
entry, so a batch pays each system's own step count, not the worst case's.  `capture()` records the factorisations and solves
of all systems into one CUDA graph, forked from the capture stream into the
side streams and joined back, so independent systems run concurrently on the
GPU; `replay()` launches the whole batch with a single graph launch; `finish()`
reports every system's final residual.

Shapes: the number of partitions p and the block size KB of each system.  The
default rule takes partitions of about 4096 rows (p = max(2, n // 4096), every
partition longer than k) and the smallest block that holds k; `autotune`
times candidate shapes on copies of a representative system of each (k, size
class) running together in one graph (enough to fill the GPU), and keeps the
one with the highest throughput when it beats the default rule clearly.
"""
from __future__ import annotations

import math
from typing import Callable, Dict, List, Optional, Sequence, Tuple

from .solver import LRSpike

Shape = Tuple[int, int]  # (p, block)


def min_block(k: int) -> int:
    kb = 8
    while kb < k:
        kb *= 2
    return kb


def partitions_for(n: int, k: int, rows: int) -> int:
    """p for partitions of about `rows` rows, at least 1, every n_i > k."""
    p = max(1, n // rows)
    while p > 1 and n // p <= k:
        p -= 1
    return p


def default_shape(n: int, k: int) -> Shape:
    """About 4096 rows per partition (at least two partitions when they fit)
    and the smallest block >= k."""
    p = max(2, n // 4096)
    while p > 1 and n // p <= k:
        p -= 1
    return p, min_block(k)


def candidate_shapes(n: int, k: int) -> List[Shape]:
    """Partitions of 1K..32K rows, block sizes KB_min and 2 KB_min (<= 64)."""
    blocks = [b for b in (min_block(k), 2 * min_block(k)) if b <= 64]
    out = []
    for rows in (1024, 2048, 4096, 8192, 16384, 32768):
        p = partitions_for(n, k, rows)
        for b in blocks:
            if (p, b) not in out:
                out.append((p, b))
    return out


def size_class(n: int) -> int:
    """Systems whose n falls in the same power-of-two interval share a shape."""
    return int(math.floor(math.log2(n)))


class BatchSolver:
    """systems: list of (band (2k+1, n) float64 device tensor, f (nrhs, n) or
    (n,) float64 device tensor, k).  shapes: one (p, block) per system, or
    None for the default rule.  Keyword options go to every LRSpike handle
    (precision, r_of_k, iterations = refinement steps, tol)."""

    def __init__(self, systems: Sequence, shapes: Optional[Sequence[Shape]] = None, precision: str = "fp32",
                 iterations: int = 6, tol: float = 1e-10, r_of_k: Callable[[int], int] = lambda k: max(1, k // 4),
                 streams: int = 32, reduced: str = "truncated"):
        import torch
        self.torch = torch
        self.systems = list(systems)
        self.shapes = list(shapes) if shapes is not None else [
            default_shape(b.shape[1], k) for b, _, k in self.systems]
        self.pool = [torch.cuda.Stream() for _ in range(min(streams, len(self.systems)))]
        self.handles, self.x = [], []
        for idx, ((band, f, k), (p, block)) in enumerate(zip(self.systems, self.shapes)):
            n = band.shape[1]
            F = f.unsqueeze(0) if f.dim() == 1 else f
            r = min(r_of_k(k), k) if p > 1 else 0
            s = LRSpike(n, k, p, r, precision=precision, reduced=reduced, outer="ir", tol=tol,
                        max_iter=iterations, max_nrhs=F.shape[0], graph_safe=True, block=block,
                        stream=self.pool[idx % len(self.pool)])
            self.handles.append(s)
            self.x.append(torch.empty_like(F))
        self.graph = None

    def _enqueue(self):
        for (band, f, _), s, x in zip(self.systems, self.handles, self.x):
            F = f.unsqueeze(0) if f.dim() == 1 else f
            s.factor(band)
            s.solve(F, x)

    def run_eager(self):
        """The same work without a graph (stream-ordered launches)."""
        torch = self.torch
        cur = torch.cuda.current_stream()
        for st in self.pool:
            st.wait_stream(cur)
        self._enqueue()
        for st in self.pool:
            cur.wait_stream(st)

    def capture(self):
        """Records every factorisation and solve into one CUDA graph: the side
        streams fork from the capture stream and join back into it."""
        torch = self.torch
        self.run_eager()                       # first use outside capture (kernel attributes, modules)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream()
        with torch.cuda.graph(g, stream=cap):
            for st in self.pool:
                st.wait_stream(cap)
            self._enqueue()
            for st in self.pool:
                cap.wait_stream(st)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def finish(self, allow_unconverged: bool = False) -> List[dict]:
        out = []
        for s, x in zip(self.handles, self.x):
            out.append(s.finish(nrhs=x.shape[0], allow_unconverged=allow_unconverged))
        return out

    def unknowns(self) -> int:
        return sum(b.shape[1] * (f.shape[0] if f.dim() == 2 else 1) for b, f, _ in self.systems)

    def close(self):
        self.graph = None
        for s in self.handles:
            s.close()
        self.handles = []


def autotune(classes: Dict[Tuple[int, int], Tuple], precision: str = "fp32", iterations: int = 6,
             reps: int = 3, tol: float = 1e-10,
             r_of_k: Callable[[int], int] = lambda k: max(1, k // 4), max_copies: int = 8,
             margin: float = 0.05) -> Dict[Tuple[int, int], Shape]:
    """classes: {(k, size class): (band, f) of a representative system}.

    A batch keeps the GPU full, so the objective is throughput, not one
    system's latency: for every class and candidate shape (the default rule's
    shape included), copies of the representative system are captured into
    one graph the way a batch runs them (side streams, concurrently), enough
    copies for about two partitions per SM (at most `max_copies`), and the
    replays are timed with CUDA events (median of `reps` after one warm-up).
    The shape with the least time per solved unknown wins; it replaces the
    default rule only when it is at least `margin` faster."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    best = {}
    for (k, cls), (band, f) in classes.items():
        n = band.shape[1]
        d = default_shape(n, k)
        cands = candidate_shapes(n, k)
        if d not in cands:
            cands.append(d)
        timings = {}
        for p, block in cands:
            copies = max(2, min(max_copies, -(-2 * sms // p)))
            bs = BatchSolver([(band, f, k)] * copies, shapes=[(p, block)] * copies, precision=precision,
                             iterations=iterations, tol=tol, r_of_k=r_of_k, streams=copies)
            try:
                bs.capture()
                ts = []
                for rep in range(reps + 1):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    bs.replay()
                    e1.record()
                    torch.cuda.synchronize()
                    if rep:
                        ts.append(e0.elapsed_time(e1))
                infos = bs.finish(allow_unconverged=True)
                if all(i["converged"] for i in infos):
                    timings[(p, block)] = sorted(ts)[len(ts) // 2] / (copies * n)
            finally:
                bs.close()
        if not timings:
            best[(k, cls)] = d
            continue
        shape = min(timings, key=timings.get)
        if d in timings and timings[shape] > (1.0 - margin) * timings[d]:
            shape = d
        best[(k, cls)] = shape
    return best
