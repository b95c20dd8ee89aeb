"""ctypes binding of libpt.so with the C ABI's names (include/pt.h).

Argument marshalling only: every step of a transfer runs in the library's
CUDA kernels.  Pointers are passed as Python ints (``tensor.data_ptr()``
or ``ndarray.ctypes.data``).  Each call raises :class:`PtError` when the
library returns a status other than ``PT_OK``.  If ``libpt.so`` has not
been built, importing this module raises ``ImportError``: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence, Tuple

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpt.so")

PT_OK, PT_ERR_INVALID, PT_ERR_OOM, PT_ERR_CUDA, PT_ERR_STATE, PT_ERR_TIMEOUT, PT_ERR_UNSUPPORTED = range(7)
PT_I32, PT_I64 = 0, 1
PT_MEM_DEVICE, PT_MEM_HOST = 0, 1
STATUS_NAMES = ["PT_OK", "PT_ERR_INVALID", "PT_ERR_OOM", "PT_ERR_CUDA", "PT_ERR_STATE", "PT_ERR_TIMEOUT",
                "PT_ERR_UNSUPPORTED"]


class PtError(RuntimeError):
    def __init__(self, status: int, func: str, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{func}: {name}: {msg}")


class pt_filter_cfg(C.Structure):
    _fields_ = [("bits_per_key", C.c_int32), ("k", C.c_int32), ("block_bits", C.c_int32),
                ("reserved", C.c_int32), ("seed", C.c_uint64)]


class pt_column(C.Structure):
    _fields_ = [("data", C.c_void_p), ("dtype", C.c_int32), ("mem", C.c_int32)]


class pt_edge(C.Structure):
    _fields_ = [("t0", C.c_int32), ("ncols", C.c_int32), ("c0", C.c_int32 * 2), ("t1", C.c_int32),
                ("c1", C.c_int32 * 2), ("flags", C.c_uint32)]


class pt_visit_stats(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("survivors", C.c_int64), ("probe_sectors", C.c_int64),
                ("build_sectors", C.c_int64), ("filter_bytes", C.c_int64), ("n_in", C.c_int32),
                ("n_out", C.c_int32), ("has_input_bitmap", C.c_int32), ("first_probe", C.c_int32),
                ("first_probe_sectors", C.c_int64)]


class pt_launch_time(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pass_", C.c_int32), ("table", C.c_int32), ("reserved", C.c_int32),
                ("start_ms", C.c_double), ("ms", C.c_double)]


class pt_kernel_times(C.Structure):
    _fields_ = [("first_ms", C.c_double), ("scan_ms", C.c_double), ("build_ms", C.c_double),
                ("first_launches", C.c_int32), ("scan_launches", C.c_int32), ("build_pairs", C.c_int32),
                ("reserved", C.c_int32)]


class pt_static_probe(C.Structure):
    _fields_ = [("col", pt_column * 2), ("ncols", C.c_int32), ("reserved", C.c_int32), ("filter", C.c_void_p),
                ("nblocks", C.c_void_p)]


class pt_static_build(C.Structure):
    _fields_ = [("col", pt_column * 2), ("ncols", C.c_int32), ("reserved", C.c_int32), ("filter", C.c_void_p),
                ("capacity_blocks", C.c_int64), ("probe_rows", C.c_int64), ("nblocks_out", C.c_void_p)]


PT_STATIC_MAX_ROWS = 1 << 20

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built (python -m paper_2307_15255_b300.build); "
                      "there is no non-CUDA fallback")

lib = C.CDLL(LIB_PATH)

_P = C.c_void_p
_SIGS = {
    "pt_abi_version": (C.c_uint32, []),
    "pt_create": (C.c_int, [C.POINTER(_P), C.POINTER(pt_filter_cfg), _P]),
    "pt_destroy": (C.c_int, [_P]),
    "pt_register_table": (C.c_int, [_P, C.c_int64, C.c_int32, C.POINTER(pt_column), _P, C.c_int32,
                                    C.POINTER(C.c_int32)]),
    "pt_update_table": (C.c_int, [_P, C.c_int32, C.POINTER(pt_column), _P, C.c_int32]),
    "pt_set_join_graph": (C.c_int, [_P, C.c_int32, C.POINTER(pt_edge)]),
    "pt_plan": (C.c_int, [_P, _P, C.POINTER(C.c_int64)]),
    "pt_run_forward": (C.c_int, [_P]),
    "pt_run_backward": (C.c_int, [_P]),
    "pt_run_transfer": (C.c_int, [_P]),
    "pt_set_graph_mode": (C.c_int, [_P, C.c_int32]),
    "pt_get_survivors": (C.c_int, [_P, C.c_int32, _P, C.POINTER(C.c_int64)]),
    "pt_get_pass_survivors": (C.c_int, [_P, C.c_int32, C.c_int32, _P, C.POINTER(C.c_int64)]),
    "pt_get_filter": (C.c_int, [_P, C.c_int32, C.c_int32, _P, C.POINTER(C.c_int64)]),
    "pt_get_visit_stats": (C.c_int, [_P, C.c_int32, C.c_int32, C.POINTER(pt_visit_stats)]),
    "pt_set_launch": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32]),
    "pt_set_kernel_timing": (C.c_int, [_P, C.c_int32]),
    "pt_set_cluster": (C.c_int, [_P, C.c_int32]),
    "pt_set_first_probe": (C.c_int, [_P, C.c_int32]),
    "pt_set_first_probe_ctas": (C.c_int, [_P, C.c_int32]),
    "pt_set_probe_order": (C.c_int, [_P, C.c_int32]),
    "pt_set_schedule": (C.c_int, [_P, C.c_int32]),
    "pt_set_early_scan": (C.c_int, [_P, C.c_int32]),
    "pt_set_dependent_launch": (C.c_int, [_P, C.c_int32]),
    "pt_join_count": (C.c_int, [_P, _P]),
    "pt_set_streams": (C.c_int, [_P, C.c_int32]),
    "pt_get_kernel_times": (C.c_int, [_P, C.POINTER(pt_kernel_times)]),
    "pt_get_launch_times": (C.c_int, [_P, C.c_int32, C.POINTER(pt_launch_time), C.POINTER(C.c_int32)]),
    "pt_get_kernel_time": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
    "pt_get_launch_count": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "pt_plan_graph": (C.c_int, [C.c_int32, _P, C.c_int32, C.POINTER(pt_edge), _P, _P, _P, _P]),
    "pt_last_error": (C.c_char_p, [_P]),
    "pt_visit_static": (C.c_int, [C.POINTER(pt_filter_cfg), _P, C.c_int64, _P, C.c_int32,
                                  C.POINTER(pt_static_probe), C.c_int32, C.POINTER(pt_static_build), _P, _P]),
    "pt_server_create": (C.c_int, [C.POINTER(_P), C.POINTER(pt_filter_cfg), C.c_int64, C.c_int32, C.c_int32]),
    "pt_server_register_table": (C.c_int, [_P, C.c_int64, C.c_int32, C.POINTER(pt_column), C.POINTER(C.c_int32)]),
    "pt_server_start": (C.c_int, [_P]),
    "pt_server_submit": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_int32), C.POINTER(_P), C.c_int32, C.c_int32,
                                   C.POINTER(pt_edge), C.POINTER(C.c_uint64)]),
    "pt_server_poll": (C.c_int, [_P, C.c_uint64, C.POINTER(C.c_int32), C.POINTER(C.c_int)]),
    "pt_server_wait": (C.c_int, [_P, C.c_uint64, C.POINTER(C.c_int)]),
    "pt_server_survivors": (C.c_int, [_P, C.c_uint64, C.c_int32, _P, C.POINTER(C.c_int64)]),
    "pt_server_release": (C.c_int, [_P, C.c_uint64]),
    "pt_server_stats": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                  C.POINTER(C.c_int64)]),
    "pt_server_reset_stats": (C.c_int, [_P]),
    "pt_server_destroy": (C.c_int, [_P]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def pt_last_error(ctx: Optional[int] = None) -> str:
    return lib.pt_last_error(ctx).decode(errors="replace")


def _check(status: int, func: str, ctx: Optional[int]) -> None:
    if status != PT_OK:
        raise PtError(status, func, pt_last_error(ctx))


def pt_abi_version() -> int:
    return int(lib.pt_abi_version())


def pt_create(bits_per_key: int = 10, k: int = 4, block_bits: int = 256, seed: int = 0,
              stream: Optional[int] = None) -> int:
    cfg = pt_filter_cfg(bits_per_key, k, block_bits, 0, seed)
    out = _P()
    _check(lib.pt_create(C.byref(out), C.byref(cfg), stream), "pt_create", None)
    return out.value


def pt_destroy(ctx: int) -> None:
    _check(lib.pt_destroy(ctx), "pt_destroy", None)


def _columns(cols: Sequence[Tuple[int, int, int]]):
    arr = (pt_column * len(cols))()
    for i, (ptr, dtype, mem) in enumerate(cols):
        arr[i].data = ptr
        arr[i].dtype = dtype
        arr[i].mem = mem
    return arr


def pt_register_table(ctx: int, n_rows: int, cols: Sequence[Tuple[int, int, int]],
                      sel: Optional[int] = None, sel_mem: int = PT_MEM_DEVICE) -> int:
    """cols: (pointer, PT_I32/PT_I64, PT_MEM_DEVICE/PT_MEM_HOST) per key column."""
    arr = _columns(cols)
    tid = C.c_int32()
    _check(lib.pt_register_table(ctx, n_rows, len(cols), arr, sel, sel_mem, C.byref(tid)),
           "pt_register_table", ctx)
    return tid.value


def pt_update_table(ctx: int, table_id: int, cols: Sequence[Tuple[int, int, int]],
                    sel: Optional[int] = None, sel_mem: int = PT_MEM_DEVICE) -> None:
    arr = _columns(cols)
    _check(lib.pt_update_table(ctx, table_id, arr, sel, sel_mem), "pt_update_table", ctx)


def _edges(edges) -> "C.Array":
    arr = (pt_edge * max(len(edges), 1))()
    for i, e in enumerate(edges):
        t0, c0, t1, c1 = e[:4]
        arr[i].t0 = t0
        arr[i].t1 = t1
        arr[i].ncols = len(c0)
        for j in range(len(c0)):
            arr[i].c0[j] = c0[j]
            arr[i].c1[j] = c1[j]
        arr[i].flags = e[4] if len(e) > 4 else 0
    return arr


def pt_set_join_graph(ctx: int, edges: Sequence[tuple]) -> None:
    """edges: (t0, (cols of t0), t1, (cols of t1)[, flags])."""
    _check(lib.pt_set_join_graph(ctx, len(edges), _edges(edges)), "pt_set_join_graph", ctx)


def pt_plan(ctx: int, n_tables: int) -> Tuple[List[int], int]:
    order = (C.c_int32 * n_tables)()
    mem = C.c_int64()
    _check(lib.pt_plan(ctx, C.cast(order, _P), C.byref(mem)), "pt_plan", ctx)
    return list(order), mem.value


def pt_run_forward(ctx: int) -> None:
    _check(lib.pt_run_forward(ctx), "pt_run_forward", ctx)


def pt_run_backward(ctx: int) -> None:
    _check(lib.pt_run_backward(ctx), "pt_run_backward", ctx)


def pt_run_transfer(ctx: int) -> None:
    _check(lib.pt_run_transfer(ctx), "pt_run_transfer", ctx)


def pt_set_graph_mode(ctx: int, on: bool) -> None:
    _check(lib.pt_set_graph_mode(ctx, int(on)), "pt_set_graph_mode", ctx)


def pt_get_survivors(ctx: int, table_id: int, bitmap_out: Optional[int]) -> int:
    cnt = C.c_int64()
    _check(lib.pt_get_survivors(ctx, table_id, bitmap_out, C.byref(cnt)), "pt_get_survivors", ctx)
    return cnt.value


def pt_get_pass_survivors(ctx: int, pass_: int, table_id: int, bitmap_out: Optional[int]) -> int:
    cnt = C.c_int64()
    _check(lib.pt_get_pass_survivors(ctx, pass_, table_id, bitmap_out, C.byref(cnt)),
           "pt_get_pass_survivors", ctx)
    return cnt.value


def pt_get_filter(ctx: int, pass_: int, edge_id: int, words_out: Optional[int]) -> int:
    nb = C.c_int64()
    _check(lib.pt_get_filter(ctx, pass_, edge_id, words_out, C.byref(nb)), "pt_get_filter", ctx)
    return nb.value


def pt_get_visit_stats(ctx: int, pass_: int, table_id: int) -> dict:
    s = pt_visit_stats()
    _check(lib.pt_get_visit_stats(ctx, pass_, table_id, C.byref(s)), "pt_get_visit_stats", ctx)
    return {f: getattr(s, f) for f, _ in pt_visit_stats._fields_ if f != "reserved"}


def pt_set_launch(ctx: int, threads: int, smem_filter_bytes: int, ctas_per_sm: int = 0) -> None:
    _check(lib.pt_set_launch(ctx, threads, smem_filter_bytes, ctas_per_sm), "pt_set_launch", ctx)


def pt_set_cluster(ctx: int, max_cluster: int) -> None:
    _check(lib.pt_set_cluster(ctx, max_cluster), "pt_set_cluster", ctx)


def pt_set_kernel_timing(ctx: int, on: bool) -> None:
    _check(lib.pt_set_kernel_timing(ctx, int(on)), "pt_set_kernel_timing", ctx)


def pt_get_kernel_time(ctx: int) -> dict:
    sm, om = C.c_double(), C.c_double()
    sn, on = C.c_int32(), C.c_int32()
    _check(lib.pt_get_kernel_time(ctx, C.byref(sm), C.byref(sn), C.byref(om), C.byref(on)),
           "pt_get_kernel_time", ctx)
    return {"scan_ms": sm.value, "scan_launches": sn.value, "other_ms": om.value,
            "other_launches": on.value}


def pt_get_kernel_times(ctx: int) -> dict:
    t = pt_kernel_times()
    _check(lib.pt_get_kernel_times(ctx, C.byref(t)), "pt_get_kernel_times", ctx)
    return {f: getattr(t, f) for f, _ in pt_kernel_times._fields_ if f != "reserved"}


def pt_get_launch_times(ctx: int) -> list:
    n = C.c_int32()
    _check(lib.pt_get_launch_times(ctx, 0, None, C.byref(n)), "pt_get_launch_times", ctx)
    arr = (pt_launch_time * max(n.value, 1))()
    _check(lib.pt_get_launch_times(ctx, n.value, arr, C.byref(n)), "pt_get_launch_times", ctx)
    kinds = {0: "scan", 1: "build", 2: "first"}
    return [{"kind": kinds[t.kind], "pass": t.pass_, "table": t.table, "start_ms": t.start_ms, "ms": t.ms}
            for t in arr[:n.value]]


def pt_set_streams(ctx: int, streams: int) -> None:
    _check(lib.pt_set_streams(ctx, streams), "pt_set_streams", ctx)


def pt_set_first_probe(ctx: int, enable: bool) -> None:
    _check(lib.pt_set_first_probe(ctx, int(enable)), "pt_set_first_probe", ctx)


def pt_set_first_probe_ctas(ctx: int, ctas_per_sm: int) -> None:
    _check(lib.pt_set_first_probe_ctas(ctx, int(ctas_per_sm)), "pt_set_first_probe_ctas", ctx)


def pt_join_count(ctx: int) -> int:
    """Size of the join of the survivors (see include/pt.h)."""
    n = C.c_uint64()
    _check(lib.pt_join_count(ctx, C.byref(n)), "pt_join_count", ctx)
    return n.value


PT_ORDER_LEVEL_LIP, PT_ORDER_LIP, PT_ORDER_EDGE = 0, 1, 2
PT_SCHEDULE_TRANSFER, PT_SCHEDULE_ONE_HOP = 0, 1


def pt_set_early_scan(ctx: int, enable: bool) -> None:
    _check(lib.pt_set_early_scan(ctx, 1 if enable else 0), "pt_set_early_scan", ctx)


def pt_set_dependent_launch(ctx: int, enable: bool) -> None:
    _check(lib.pt_set_dependent_launch(ctx, 1 if enable else 0), "pt_set_dependent_launch", ctx)


def pt_set_schedule(ctx: int, schedule: int) -> None:
    _check(lib.pt_set_schedule(ctx, int(schedule)), "pt_set_schedule", ctx)


def pt_set_probe_order(ctx: int, order: int) -> None:
    _check(lib.pt_set_probe_order(ctx, int(order)), "pt_set_probe_order", ctx)


def pt_get_launch_count(ctx: int) -> int:
    n = C.c_int64()
    _check(lib.pt_get_launch_count(ctx, C.byref(n)), "pt_get_launch_count", ctx)
    return n.value


def pt_visit_static(n_rows: int, in_bits: Optional[int], probes: Sequence[tuple], builds: Sequence[tuple],
                    out_bits: int, count_out: Optional[int], bits_per_key: int = 10, k: int = 4,
                    block_bits: int = 256, seed: int = 0, stream: Optional[int] = None) -> None:
    """One visit with no allocation (see include/pt.h).

    probes: (cols, filter_ptr, nblocks_ptr) with cols a list of (ptr, dtype);
    builds: (cols, filter_ptr, capacity_blocks, probe_rows, nblocks_out_ptr).
    All pointers are device pointers.
    """
    cfg = pt_filter_cfg(bits_per_key, k, block_bits, 0, seed)
    pa = (pt_static_probe * max(len(probes), 1))()
    for i, (cols, fptr, nbptr) in enumerate(probes):
        pa[i].ncols = len(cols)
        for j, (ptr, dt) in enumerate(cols):
            pa[i].col[j].data, pa[i].col[j].dtype, pa[i].col[j].mem = ptr, dt, PT_MEM_DEVICE
        pa[i].filter, pa[i].nblocks = fptr, nbptr
    ba = (pt_static_build * max(len(builds), 1))()
    for i, (cols, fptr, cap, prows, nbout) in enumerate(builds):
        ba[i].ncols = len(cols)
        for j, (ptr, dt) in enumerate(cols):
            ba[i].col[j].data, ba[i].col[j].dtype, ba[i].col[j].mem = ptr, dt, PT_MEM_DEVICE
        ba[i].filter, ba[i].capacity_blocks, ba[i].probe_rows, ba[i].nblocks_out = fptr, cap, prows, nbout
    _check(lib.pt_visit_static(C.byref(cfg), stream, n_rows, in_bits, len(probes), pa, len(builds), ba, out_bits,
                               count_out), "pt_visit_static", None)


def pt_plan_graph(n_rows: Sequence[int], edges: Sequence[tuple]) -> dict:
    """Host-only planner: orientation, forward order and levels (no GPU needed)."""
    nt, ne = len(n_rows), len(edges)
    nr = (C.c_int64 * nt)(*n_rows)
    src = (C.c_int32 * max(ne, 1))()
    dst = (C.c_int32 * max(ne, 1))()
    order = (C.c_int32 * nt)()
    level = (C.c_int32 * nt)()
    _check(lib.pt_plan_graph(nt, C.cast(nr, _P), ne, _edges(edges), C.cast(src, _P), C.cast(dst, _P),
                             C.cast(order, _P), C.cast(level, _P)), "pt_plan_graph", None)
    return {"src": list(src)[:ne], "dst": list(dst)[:ne], "order": list(order), "level": list(level)}


# ---- serving ---------------------------------------------------------------

def pt_server_create(bits_per_key: int = 10, k: int = 4, block_bits: int = 256, seed: int = 0,
                     arena_bytes: int = 1 << 30, max_batch: int = 16, max_inflight: int = 2) -> int:
    cfg = pt_filter_cfg(bits_per_key, k, block_bits, 0, seed)
    out = _P()
    _check(lib.pt_server_create(C.byref(out), C.byref(cfg), arena_bytes, max_batch, max_inflight),
           "pt_server_create", None)
    return out.value


def pt_server_register_table(srv: int, n_rows: int, cols: Sequence[Tuple[int, int, int]]) -> int:
    arr = _columns(cols)
    tid = C.c_int32()
    _check(lib.pt_server_register_table(srv, n_rows, len(cols), arr, C.byref(tid)), "pt_server_register_table", None)
    return tid.value


def pt_server_start(srv: int) -> None:
    _check(lib.pt_server_start(srv), "pt_server_start", None)


def pt_server_submit(srv: int, table_ids: Sequence[int], sel_ptrs: Sequence[Optional[int]],
                     edges: Sequence[tuple], sel_mem: int = PT_MEM_HOST) -> int:
    """sel_ptrs: addresses of uint32 bitmaps (or None) per instance: host memory
    (copied before returning) or device memory (borrowed until done)."""
    n = len(table_ids)
    ids = (C.c_int32 * n)(*table_ids)
    sels = (_P * n)(*[p for p in sel_ptrs])
    t = C.c_uint64()
    _check(lib.pt_server_submit(srv, n, ids, sels, sel_mem, len(edges), _edges(edges), C.byref(t)),
           "pt_server_submit", None)
    return t.value


def pt_server_poll(srv: int, ticket: int) -> Tuple[bool, int]:
    done, res = C.c_int32(), C.c_int()
    _check(lib.pt_server_poll(srv, ticket, C.byref(done), C.byref(res)), "pt_server_poll", None)
    return bool(done.value), res.value


def pt_server_wait(srv: int, ticket: int) -> int:
    res = C.c_int()
    _check(lib.pt_server_wait(srv, ticket, C.byref(res)), "pt_server_wait", None)
    return res.value


def pt_server_survivors(srv: int, ticket: int, inst: int, bitmap_out: Optional[int]) -> int:
    c = C.c_int64()
    _check(lib.pt_server_survivors(srv, ticket, inst, bitmap_out, C.byref(c)), "pt_server_survivors", None)
    return c.value


def pt_server_release(srv: int, ticket: int) -> None:
    _check(lib.pt_server_release(srv, ticket), "pt_server_release", None)


def pt_server_stats(srv: int) -> dict:
    p50, p99, qps = C.c_double(), C.c_double(), C.c_double()
    n = C.c_int64()
    _check(lib.pt_server_stats(srv, C.byref(p50), C.byref(p99), C.byref(qps), C.byref(n)), "pt_server_stats", None)
    return {"p50_ms": p50.value, "p99_ms": p99.value, "qps": qps.value, "completed": n.value}


def pt_server_reset_stats(srv: int) -> None:
    _check(lib.pt_server_reset_stats(srv), "pt_server_reset_stats", None)


def pt_server_destroy(srv: int) -> None:
    _check(lib.pt_server_destroy(srv), "pt_server_destroy", None)
