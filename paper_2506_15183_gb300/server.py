"""Python binding of the serving loop (``include/yoro_server.h``): argument marshalling only.

Every stream's resident slots are device memory owned by the library; ``Server.slot``
returns torch views of them (zero-copy, through ``__cuda_array_interface__``), so a
renderer writes the left eye straight into a slot and reads the right eye from it.
"""
from __future__ import annotations

import ctypes

import torch

from . import YoroError, load_library


class Completion(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_int), ("slot", ctypes.c_int), ("tag", ctypes.c_ulonglong),
                ("submit_ns", ctypes.c_longlong), ("launch_ns", ctypes.c_longlong), ("done_ns", ctypes.c_longlong),
                ("batch_frames", ctypes.c_int), ("status", ctypes.c_int), ("inpainted", ctypes.c_int)]


def _lib():
    lib = load_library()
    if not getattr(lib, "_server_typed", False):
        P, I, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
        lib.yoro_server_create.argtypes = [ctypes.c_size_t, I]
        lib.yoro_server_create.restype = P
        lib.yoro_server_destroy.argtypes = [P]
        lib.yoro_server_destroy.restype = None
        lib.yoro_server_admit.argtypes = [P, I, I, F, F, F, F, F, F, F, I]
        lib.yoro_server_admit.restype = I
        lib.yoro_server_leave.argtypes = [P, I]
        lib.yoro_server_leave.restype = I
        lib.yoro_server_slot.argtypes = [P, I, I, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                                         ctypes.POINTER(P)]
        lib.yoro_server_slot.restype = I
        lib.yoro_server_submit.argtypes = [P, I, I, ctypes.c_ulonglong]
        lib.yoro_server_submit.restype = I
        lib.yoro_server_poll.argtypes = [P, ctypes.POINTER(Completion), I]
        lib.yoro_server_poll.restype = I
        lib.yoro_server_drain.argtypes = [P, I]
        lib.yoro_server_drain.restype = I
        lib.yoro_server_memory_used.argtypes = [P]
        lib.yoro_server_memory_used.restype = ctypes.c_size_t
        lib.yoro_server_admit_ex.argtypes = [P, I, I, F, F, F, F, F, F, F, I, I]
        lib.yoro_server_admit_ex.restype = I
        lib.yoro_server_set_inpainter.argtypes = [P, P]
        lib.yoro_server_set_inpainter.restype = I
        lib.yoro_server_pause.argtypes = [P, I]
        lib.yoro_server_pause.restype = I
        lib.yoro_server_cancel.argtypes = [P, I]
        lib.yoro_server_cancel.restype = I
        lib.yoro_server_feed.argtypes = [P, I, ctypes.POINTER(P), ctypes.POINTER(P), I, ctypes.c_longlong, F,
                                         ctypes.c_ulonglong]
        lib.yoro_server_feed.restype = I
        lib.yoro_server_feed_stop.argtypes = [P]
        lib.yoro_server_feed_stop.restype = I
        lib._server_typed = True
    return lib


class _DeviceArray:
    """A device buffer the library owns, seen by torch through __cuda_array_interface__."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 2, "strides": None}


class Server:
    def __init__(self, memory_budget_bytes: int, max_batch: int = 64):
        lib = _lib()
        self._s = lib.yoro_server_create(int(memory_budget_bytes), int(max_batch))
        if not self._s:
            raise YoroError(lib.yoro_last_create_error(), "yoro_server_create")
        self._shapes = {}

    def admit(self, w, h, fx, fy, cx, cy, ipd, near=0.05, far=1000.0, slots=2, learned=False) -> int:
        """Stream id, or raises YoroError (YORO_ENOMEM when the budget is full).  learned:
        the stream's holes are repainted by the server's inpainter (set_inpainter)."""
        r = _lib().yoro_server_admit_ex(self._s, int(w), int(h), fx, fy, cx, cy, ipd, near, far, int(slots),
                                        int(bool(learned)))
        if r < 0:
            raise YoroError(-r, "yoro_server_admit")
        self._shapes[r] = (int(h), int(w))
        return r

    def leave(self, stream: int) -> None:
        st = _lib().yoro_server_leave(self._s, int(stream))
        if st != 0:
            raise YoroError(st, "yoro_server_leave")

    def slot(self, stream: int, slot: int):
        """(color uint8[H,W,4], depth float32[H,W], out_color uint8[H,W,4], out_mask uint8[H,W]) views."""
        P = ctypes.c_void_p
        c, d, o, m = P(), P(), P(), P()
        st = _lib().yoro_server_slot(self._s, int(stream), int(slot), ctypes.byref(c), ctypes.byref(d),
                                     ctypes.byref(o), ctypes.byref(m))
        if st != 0:
            raise YoroError(st, "yoro_server_slot")
        h, w = self._shapes[stream]
        dev = torch.device("cuda", torch.cuda.current_device())
        return (torch.as_tensor(_DeviceArray(c.value, (h, w, 4), "|u1"), device=dev),
                torch.as_tensor(_DeviceArray(d.value, (h, w), "<f4"), device=dev),
                torch.as_tensor(_DeviceArray(o.value, (h, w, 4), "|u1"), device=dev),
                torch.as_tensor(_DeviceArray(m.value, (h, w), "|u1"), device=dev))

    def submit(self, stream: int, slot: int, tag: int = 0) -> None:
        st = _lib().yoro_server_submit(self._s, int(stream), int(slot), int(tag))
        if st != 0:
            raise YoroError(st, "yoro_server_submit")

    def poll(self, max_records: int = 1024):
        buf = (Completion * max_records)()
        n = _lib().yoro_server_poll(self._s, buf, max_records)
        return [buf[i] for i in range(n)]

    def drain(self, timeout_ms: int = 10000) -> None:
        st = _lib().yoro_server_drain(self._s, int(timeout_ms))
        if st != 0:
            raise YoroError(st, "yoro_server_drain")

    def set_inpainter(self, inpainter) -> None:
        """An Inpainter (paper_2506_15183_gb300.unet) or None; the caller keeps it alive."""
        st = _lib().yoro_server_set_inpainter(self._s, inpainter.ptr if inpainter is not None else None)
        if st != 0:
            raise YoroError(st, "yoro_server_set_inpainter")

    def pause(self, paused: bool = True) -> None:
        st = _lib().yoro_server_pause(self._s, int(bool(paused)))
        if st != 0:
            raise YoroError(st, "yoro_server_pause")

    def cancel(self, stream: int) -> int:
        n = _lib().yoro_server_cancel(self._s, int(stream))
        if n < 0:
            raise YoroError(-n, "yoro_server_cancel")
        return n

    def feed(self, stream: int, frames, nframes: int, hz: float = 0.0, tag0: int = 0) -> None:
        """The server's feeder copies frames[i % len(frames)] = (color, depth) device tensors
        into the stream's free slots and submits them, nframes times (hz > 0: paced)."""
        n = len(frames)
        cols = (ctypes.c_void_p * n)(*[c.data_ptr() for c, _ in frames])
        deps = (ctypes.c_void_p * n)(*[d.data_ptr() for _, d in frames])
        st = _lib().yoro_server_feed(self._s, int(stream), cols, deps, n, int(nframes), float(hz), int(tag0))
        if st != 0:
            raise YoroError(st, "yoro_server_feed")

    def feed_stop(self) -> None:
        _lib().yoro_server_feed_stop(self._s)

    def memory_used(self) -> int:
        return int(_lib().yoro_server_memory_used(self._s))

    def close(self) -> None:
        if self._s:
            _lib().yoro_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass
