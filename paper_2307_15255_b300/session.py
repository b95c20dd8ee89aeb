"""A predicate-transfer context over torch tensors.

PyTorch supplies device memory and the stream; every step of the
transfer runs in libpt's kernels (see :mod:`paper_2307_15255_b300.pt`).
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import torch

from . import pt as _pt


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.int32:
        return _pt.PT_I32
    if t.dtype == torch.int64:
        return _pt.PT_I64
    raise TypeError(f"key columns must be int32 or int64 tensors, got {t.dtype}")


def _mem(t: torch.Tensor) -> int:
    return _pt.PT_MEM_DEVICE if t.is_cuda else _pt.PT_MEM_HOST


class TransferSession:
    """Tables, join graph and plan of one predicate transfer.

    ``tables``: sequence of ``(n_rows, [key column tensors], sel)`` where
    a column is a contiguous int32/int64 tensor (CUDA: borrowed; CPU:
    copied to the device, asynchronously when pinned) and ``sel`` an int32
    tensor holding the uint32 selection bitmap words, or ``None``.
    ``edges``: sequence of ``(t0, (cols of t0), t1, (cols of t1))`` or
    ``(t0, cols, t1, cols, flags)``.  ``schedule``: ``PT_SCHEDULE_TRANSFER``
    (forward and backward pass) or ``PT_SCHEDULE_ONE_HOP`` (a Bloom join:
    every filter built from its table's selection, probed once).
    """

    def __init__(self, tables: Sequence[Tuple[int, Sequence[torch.Tensor], Optional[torch.Tensor]]],
                 edges: Sequence[tuple], bits_per_key: int = 10, k: int = 4, block_bits: int = 256,
                 seed: int = 0, stream: Optional[torch.cuda.Stream] = None,
                 launch: Optional[Tuple[int, int, int]] = None, graph: bool = False,
                 cluster: Optional[int] = None, first_probe: Optional[bool] = None,
                 probe_order: Optional[int] = None, schedule: int = _pt.PT_SCHEDULE_TRANSFER):
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.block_bits = block_bits
        self.bits_per_key = bits_per_key
        self.k = k
        self.schedule = schedule
        self.col_dtypes = []
        self.ctx = _pt.pt_create(bits_per_key, k, block_bits, seed, self.stream.cuda_stream)
        self._keep: List[torch.Tensor] = []
        self.n_rows = []
        try:
            for n, cols, sel in tables:
                cols = [c.contiguous() for c in cols]
                self._keep.extend(cols)
                spec = [(c.data_ptr(), _dtype_code(c), _mem(c)) for c in cols]
                sp, sm = None, _pt.PT_MEM_DEVICE
                if sel is not None:
                    sel = sel.contiguous()
                    self._keep.append(sel)
                    sp, sm = sel.data_ptr(), _mem(sel)
                _pt.pt_register_table(self.ctx, int(n), spec, sp, sm)
                self.n_rows.append(int(n))
                self.col_dtypes.append([str(c.dtype) for c in cols])
            self.edges = [tuple(e) for e in edges]
            _pt.pt_set_join_graph(self.ctx, self.edges)
            if launch is not None:
                _pt.pt_set_launch(self.ctx, *launch)
            if cluster is not None:
                _pt.pt_set_cluster(self.ctx, cluster)
            if first_probe is not None:
                _pt.pt_set_first_probe(self.ctx, first_probe)
            if probe_order is not None:
                _pt.pt_set_probe_order(self.ctx, probe_order)
            _pt.pt_set_schedule(self.ctx, schedule)
            self.order, self.mem_bytes = _pt.pt_plan(self.ctx, len(self.n_rows))
            if graph:
                _pt.pt_set_graph_mode(self.ctx, True)
        except Exception:
            _pt.pt_destroy(self.ctx)
            self.ctx = None
            raise

    # -- running ---------------------------------------------------------
    def run(self) -> None:
        """Forward then backward pass (asynchronous on the session's stream)."""
        _pt.pt_run_transfer(self.ctx)

    def forward(self) -> None:
        _pt.pt_run_forward(self.ctx)

    def backward(self) -> None:
        _pt.pt_run_backward(self.ctx)

    def update(self, table_id: int, cols: Sequence[torch.Tensor], sel: Optional[torch.Tensor] = None) -> None:
        cols = [c.contiguous() for c in cols]
        self._keep.extend(cols)
        spec = [(c.data_ptr(), _dtype_code(c), _mem(c)) for c in cols]
        sp, sm = None, _pt.PT_MEM_DEVICE
        if sel is not None:
            self._keep.append(sel)
            sp, sm = sel.data_ptr(), _mem(sel)
        _pt.pt_update_table(self.ctx, table_id, spec, sp, sm)

    # -- results ---------------------------------------------------------
    def survivors(self, table_id: int, pass_: Optional[int] = None, out: Optional[torch.Tensor] = None):
        """(bitmap as an int32 tensor, survivor count); device tensor unless ``out`` is given."""
        nw = (self.n_rows[table_id] + 31) // 32
        if out is None:
            out = torch.empty(max(nw, 1), dtype=torch.int32, device="cuda")
        if pass_ is None:
            c = _pt.pt_get_survivors(self.ctx, table_id, out.data_ptr())
        else:
            c = _pt.pt_get_pass_survivors(self.ctx, pass_, table_id, out.data_ptr())
        return out[:nw], c

    def filter(self, pass_: int, edge_id: int) -> torch.Tensor:
        nb = _pt.pt_get_filter(self.ctx, pass_, edge_id, None)
        out = torch.empty(nb * self.block_bits // 32, dtype=torch.int32, device="cuda")
        _pt.pt_get_filter(self.ctx, pass_, edge_id, out.data_ptr())
        return out

    def stats(self, pass_: int, table_id: int) -> Optional[dict]:
        """The visit's accounting; None for a table the pass does not visit."""
        try:
            return _pt.pt_get_visit_stats(self.ctx, pass_, table_id)
        except _pt.PtError as e:
            if e.status == _pt.PT_ERR_INVALID and self.schedule == _pt.PT_SCHEDULE_ONE_HOP and pass_ == 0:
                return None
            raise

    def join_count(self) -> int:
        """Size of the join of the survivors (acyclic graphs of inner joins)."""
        return _pt.pt_join_count(self.ctx)

    def close(self) -> None:
        if self.ctx is not None:
            _pt.pt_destroy(self.ctx)
            self.ctx = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
