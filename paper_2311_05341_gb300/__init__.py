"""GB300-native brute-force incoherent dedispersion (arxiv 2311.05341).

Python binding of libdd (include/dd.h).  PyTorch supplies device memory and
streams only; every step of the transform runs in the library's CUDA kernels.

    plan = Plan(freqs_mhz, f_ref_mhz, t_samp_s, [(lo, hi, step, bin), ...], "u8")
    planes = plan.run(x)          # x: cuda tensor [n_chan][n_samp]
    # planes[r]: [n_dm_r][n_out_r] int32 (u8/u16) or float32 (f32)

Y_r[d][t] = sum_c X_r[c][t + s_r(c, d)] with the shift law of Eq. 1 and the
direct transform of Eq. 3 (Sec. 2 of the paper); see include/dd.h.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import DDError, check

__all__ = ["Plan", "DDError", "build", "DTYPES"]

DTYPES = {"u8": _lib.DD_U8, "u16": _lib.DD_U16, "f32": _lib.DD_F32, "u4": _lib.DD_U4}
# Torch element type of each dtype's buffers ("u4": packed bytes, two samples each).
_TORCH_DTYPE_NAMES = {"u8": "uint8", "u16": "uint16", "f32": "float32", "u4": "uint8"}


def _samples_per_elem(dtype: str) -> int:
    return 2 if dtype == "u4" else 1


def build(force: bool = False) -> str:
    """Compile libdd.so for sm_103a (in-tree)."""
    from . import builder
    return builder.build(force=force)


def transpose(x_tm, n_chan: int | None = None, out=None, t_begin: int = 0,
              t_end: int | None = None, stream=None):
    """Time-major cuda tensor x_tm [n_samp][stride >= n_chan] -> channel-major
    [n_chan][stride' >= n_samp] (dd_transpose); rows of `out` padded to 16 bytes."""
    import torch
    names = {"uint8": "u8", "uint16": "u16", "float32": "f32"}
    dt = names[str(x_tm.dtype).replace("torch.", "")]
    n_samp = x_tm.shape[0]
    nc = x_tm.shape[1] if n_chan is None else int(n_chan)
    if out is None:
        per = 16 // x_tm.element_size()
        out = torch.zeros((nc, (n_samp + per - 1) // per * per), dtype=x_tm.dtype,
                          device=x_tm.device)
    te = n_samp if t_end is None else int(t_end)
    check(_lib.load().dd_transpose(DTYPES[dt], x_tm.data_ptr(), x_tm.stride(0), nc,
                                   out.data_ptr(), out.stride(0), int(t_begin), te,
                                   _stream_ptr(stream)))
    return out


def dm_ranges(freqs, t_samp: float, dm_max: float, tol: float = 1.25, width: float = 0.0,
              max_bin: int = 16, max_ranges: int = 16) -> list:
    """DM ranges [(lo, hi, step, bin)] from a smearing tolerance (dd_plan_dm_ranges)."""
    f = np.ascontiguousarray(freqs, dtype=np.float64)
    arr = (_lib.Range * _lib.DD_MAX_RANGES)()
    n = ctypes.c_int32()
    check(_lib.load().dd_plan_dm_ranges(f.ctypes.data, f.size, float(t_samp), float(dm_max),
                                        float(tol), float(width), int(max_bin), int(max_ranges),
                                        ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(n)))
    return [(arr[i].dm_lo, arr[i].dm_hi, arr[i].dm_step, arr[i].bin) for i in range(n.value)]


def tile_shapes() -> list:
    """The pattern-tile shape table (dd_tile_shapes) as dicts, by index."""
    lib = _lib.load()
    n = ctypes.c_int32()
    check(lib.dd_tile_shapes(None, 0, ctypes.byref(n)))
    arr = (_lib.TileShape * n.value)()
    check(lib.dd_tile_shapes(ctypes.cast(arr, ctypes.c_void_p), n.value, ctypes.byref(n)))
    return [{f: getattr(a, f) for f, _ in _lib.TileShape._fields_} for a in arr]


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Plan:
    """A dedispersion plan: channel frequencies, sampling time and DM ranges.

    ``ranges`` is a sequence of ``(dm_lo, dm_hi, dm_step, bin)``: trial DMs
    lo, lo+step, ... (half-open, fixed step per range as in Table 2), each range
    dedispersed at time bin ``bin``.  The device tables are uploaded into a
    torch-owned workspace on ``device`` when ``upload`` is true.
    """

    def __init__(self, freqs_mhz, f_ref_mhz: float, t_samp_s: float, ranges, dtype: str = "u8",
                 device=None, upload: bool = True):
        self._lib = _lib.load()
        if dtype not in DTYPES:
            raise ValueError(f"dtype must be one of {list(DTYPES)}")
        self.dtype = dtype
        self.freqs = np.ascontiguousarray(np.asarray(freqs_mhz, dtype=np.float64))
        self.f_ref = float(f_ref_mhz)
        self.t_samp = float(t_samp_s)
        self.ranges = [tuple(r) for r in ranges]
        arr = (_lib.Range * len(self.ranges))(
            *[_lib.Range(float(a), float(b), float(c), int(d)) for a, b, c, d in self.ranges])
        handle = ctypes.c_void_p()
        check(self._lib.dd_plan_create(
            self.freqs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), self.freqs.size,
            self.f_ref, self.t_samp, arr, len(self.ranges), DTYPES[dtype], ctypes.byref(handle)))
        self._h = handle
        self.workspace = None
        if upload:
            self.upload(device)

    # -- host queries -----------------------------------------------------
    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    @property
    def n_chan(self) -> int:
        return int(self.freqs.size)

    def info(self, n_samp: int) -> dict:
        inf = _lib.PlanInfo()
        check(self._lib.dd_plan_query(self._h, int(n_samp), ctypes.byref(inf)))
        n = inf.n_ranges
        return {
            "n_chan": inf.n_chan, "n_ranges": n, "n_samp": inf.n_samp,
            "n_dm": [inf.n_dm[i] for i in range(n)], "s_max": [inf.s_max[i] for i in range(n)],
            "n_out": [inf.n_out[i] for i in range(n)],
            "out_offset": [inf.out_offset[i] for i in range(n)],
            "out_elems": inf.out_elems, "n_dm_total": inf.n_dm_total,
            "max_delay_raw": inf.max_delay_raw, "workspace_bytes": inf.workspace_bytes,
            "kernel": [{1: "generic", 2: "tiled"}[inf.kernel[i]] for i in range(n)],
            "tile_dms": [inf.tile_dms[i] for i in range(n)],
            "adjoint_kernel": {0: None, 1: "gather", 2: "pattern"}[inf.adjoint_kernel],
            "tile_shape": [inf.tile_shape[i] for i in range(n)],
            "packed_copy": [bool(inf.packed_copy[i]) for i in range(n)],
        }

    def shifts(self, r: int = 0) -> np.ndarray:
        """int32 [n_dm][n_chan] shift table of range r (host copy)."""
        n_dm = self.info(0)["n_dm"][r]
        out = np.empty((n_dm, self.n_chan), dtype=np.int32)
        check(self._lib.dd_plan_shifts(self._h, int(r), out.ctypes.data))
        return out

    def set_tile(self, r: int, tile, device=None):
        """Pick the register tile of range r and re-upload.

        tile: DMs per lane of the offset tile (8, 6, 4, 2, 1), "pattern"
        (DD_TILE_PATTERN), "packed" (DD_TILE_PACKED: the pattern tile on a
        packed copy of the input, made in scratch by run()), or 0 for the
        automatic choice.
        """
        code = {"pattern": _lib.DD_TILE_PATTERN, "packed": _lib.DD_TILE_PACKED}.get(tile, tile)
        code = int(code)
        check(self._lib.dd_plan_set_tile(self._h, int(r), code))
        if self.workspace is not None:
            self.upload(self.workspace.device if device is None else device)
        return self

    def set_tile_shape(self, r: int, tile, shape: int, device=None):
        """Range r on the pattern tile ("pattern") or the packed tile
        ("packed") with one explicit shape of tile_shapes() (-1: automatic);
        re-uploads."""
        code = {"pattern": _lib.DD_TILE_PATTERN, "packed": _lib.DD_TILE_PACKED}[tile]
        check(self._lib.dd_plan_set_tile_shape(self._h, int(r), code, int(shape)))
        if self.workspace is not None:
            self.upload(self.workspace.device if device is None else device)
        return self

    # -- device -----------------------------------------------------------
    def upload(self, device=None, stream=None):
        import torch
        dev = torch.device("cuda" if device is None else device)
        nbytes = max(int(self.info(0)["workspace_bytes"]), 16)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        check(self._lib.dd_plan_upload(self._h, self.workspace.data_ptr(), nbytes,
                                       _stream_ptr(stream)))
        torch.cuda.current_stream(dev).synchronize() if stream is None else stream.synchronize()
        return self

    def out_dtype(self):
        import torch
        return torch.float32 if self.dtype == "f32" else torch.int32

    def empty_output(self, n_samp: int, device=None):
        import torch
        inf = self.info(n_samp)
        dev = self.workspace.device if device is None else device
        return torch.empty(max(inf["out_elems"], 4), dtype=self.out_dtype(), device=dev)

    def split(self, flat, n_samp: int):
        """Views of a flat output buffer as per-range [n_dm][n_out] planes."""
        inf = self.info(n_samp)
        return [flat[o:o + nd * no].view(nd, no)
                for o, nd, no in zip(inf["out_offset"], inf["n_dm"], inf["n_out"])]

    def run(self, x, out=None, n_samp: int | None = None, stream=None, segments: int = 8):
        """Forward transform of a cuda tensor x [n_chan][stride] -> list of planes.

        For "u4" plans x holds packed bytes [n_chan][stride / 2].  Ranges with a
        packed copy (info()["packed_copy"]) run from packed words in scratch
        from torch's caching allocator: a ring of `segments` time segments
        (dd_plan_packed_scratch_bytes; about 2 / segments of the full copy),
        1 for the full copy, 0 for none (the automatic tiles then unpack the
        input themselves; DD_TILE_PACKED ranges always get their copies)."""
        self._check_input(x)
        per = _samples_per_elem(self.dtype)
        n = x.shape[1] * per if n_samp is None else int(n_samp)
        if out is None:
            out = self.empty_output(n, x.device)
        scratch = self._input_scratch(n, x.device, segments)
        check(self._lib.dd_run_scratch(
            self._h, x.data_ptr(), x.stride(0) * per, n, out.data_ptr(),
            None if scratch is None else scratch.data_ptr(),
            0 if scratch is None else scratch.numel(), _stream_ptr(stream)))
        if scratch is not None and stream is not None:
            scratch.record_stream(stream)
        return self.split(out, n)

    def _input_scratch(self, n_samp: int, device, segments: int = 0):
        """Device scratch for the packed copies of a run (None when it needs
        none), from torch's caching allocator for each run: the DD_TILE_PACKED
        ranges' copies, and with segments > 0 the ring (or, where the plan has
        no ring, the full copies) of every range with a packed copy."""
        import torch
        need = self.input_scratch_bytes(n_samp)
        if segments > 0 and any(self.info(n_samp)["packed_copy"]):
            try:
                need = max(need, self.packed_scratch_bytes(n_samp, segments))
            except DDError as err:  # no ring for this plan: the full copies
                if err.status != _lib.DD_ERR_UNSUPPORTED:
                    raise
                need = max(need, self.packed_scratch_bytes(n_samp, 1))
        if need == 0:
            return None
        return torch.empty(int(need), dtype=torch.uint8, device=device)

    def packed_scratch_bytes(self, n_samp: int, segments: int = 16) -> int:
        """Scratch bytes with which every range with a packed copy runs from
        packed words: a ring of `segments` time segments, or the full copies
        for segments == 1 (dd_plan_packed_scratch_bytes)."""
        need = ctypes.c_size_t(0)
        check(self._lib.dd_plan_packed_scratch_bytes(self._h, int(n_samp), int(segments),
                                                     ctypes.byref(need)))
        return int(need.value)

    def run_window(self, x, n_keep, out=None, n_samp: int | None = None, stream=None,
                   scratch=None):
        """The first n_keep[r] outputs of every range r (dd_run_window): a list of
        [n_dm_r][n_keep[r]] planes in one flat buffer `out` (allocated if None).
        scratch: device uint8 tensor for packed-tile ranges (allocated per call
        from torch's caching allocator if None and the plan needs it)."""
        import torch
        self._check_input(x)
        per = _samples_per_elem(self.dtype)
        n = x.shape[1] * per if n_samp is None else int(n_samp)
        keep = [int(k) for k in n_keep]
        n_dm = self.info(0)["n_dm"]
        total = sum(a * b for a, b in zip(n_dm, keep))
        if out is None:
            out = torch.empty(max(total, 4), dtype=self.out_dtype(), device=x.device)
        if scratch is None:
            scratch = self._input_scratch(n, x.device)
        arr = (ctypes.c_int64 * len(keep))(*keep)
        check(self._lib.dd_run_window(
            self._h, x.data_ptr(), x.stride(0) * per, n, arr, out.data_ptr(),
            None if scratch is None else scratch.data_ptr(),
            0 if scratch is None else scratch.numel(), _stream_ptr(stream)))
        if scratch is not None and stream is not None:
            scratch.record_stream(stream)
        planes, off = [], 0
        for a, b in zip(n_dm, keep):
            planes.append(out[off:off + a * b].view(a, b))
            off += a * b
        return planes

    def input_scratch_bytes(self, n_samp: int) -> int:
        """Device scratch bytes of the packed-tile ranges (0 without any)."""
        need = ctypes.c_size_t(0)
        check(self._lib.dd_plan_input_scratch_bytes(self._h, int(n_samp), ctypes.byref(need)))
        return int(need.value)

    def set_wait_limit(self, max_polls: int = 0, hold_stage: int = -1):
        """Bound of the kernels' pipeline waits (0: default) and the timeout
        test hook (dd_plan_set_wait_limit)."""
        check(self._lib.dd_plan_set_wait_limit(self._h, int(max_polls), int(hold_stage)))
        return self

    def device_status(self, stream=None):
        """Raises DDError(DD_ERR_TIMEOUT) if a bounded device wait of an earlier
        run gave up (dd_plan_device_status); synchronises the stream."""
        check(self._lib.dd_plan_device_status(self._h, _stream_ptr(stream)))

    def run_raw(self, x_ptr: int, stride: int, n_samp: int, out_ptr: int, stream_ptr: int,
                scratch=None):
        """Forward transform on raw device pointers (no checks beyond the
        library's); scratch: a device uint8 tensor for packed-tile ranges."""
        check(self._lib.dd_run_scratch(self._h, x_ptr, stride, n_samp, out_ptr,
                                       None if scratch is None else scratch.data_ptr(),
                                       0 if scratch is None else scratch.numel(), stream_ptr))

    def run_adjoint(self, ybar_flat, n_samp: int, xbar=None, stream=None):
        """Adjoint of run() for f32 plans: flat cotangent -> [n_chan][n_samp] float32."""
        import torch
        if xbar is None:
            stride = (n_samp + 3) // 4 * 4
            xbar = torch.empty((self.n_chan, stride), dtype=torch.float32,
                               device=ybar_flat.device)
        need = ctypes.c_size_t(0)
        check(self._lib.dd_adjoint_scratch_bytes(self._h, int(n_samp), ctypes.byref(need)))
        scratch = (torch.empty(int(need.value), dtype=torch.uint8, device=ybar_flat.device)
                   if need.value else None)
        check(self._lib.dd_run_adjoint_scratch(
            self._h, ybar_flat.data_ptr(), xbar.data_ptr(), int(n_samp), xbar.stride(0),
            None if scratch is None else scratch.data_ptr(), int(need.value),
            _stream_ptr(stream)))
        if scratch is not None:
            # The scratch stays in use until the call's work on the stream ends.
            scratch.record_stream(torch.cuda.current_stream(ybar_flat.device)
                                  if stream is None else stream)
        return xbar[:, :n_samp]

    def run_host_tmajor(self, h_in, h_out, d_tm_stage, d_cm_stage, d_out_stage,
                        n_samp: int | None = None, stream=None):
        """Host-to-host forward from time-major input h_in [n_samp][stride >= n_chan]
        (pinned), staged in d_tm_stage (same shape) and transposed into d_cm_stage
        [n_chan][stride >= n_samp]."""
        n = h_in.shape[0] if n_samp is None else int(n_samp)
        check(self._lib.dd_run_host_tmajor(self._h, h_in.data_ptr(), h_in.stride(0), n,
                                           h_out.data_ptr(), d_tm_stage.data_ptr(),
                                           d_cm_stage.data_ptr(), d_cm_stage.stride(0),
                                           d_out_stage.data_ptr(), _stream_ptr(stream)))

    def run_host(self, h_in, h_out, d_in_stage, d_out_stage, n_samp: int | None = None,
                 stream=None, packed: bool = True):
        """Host-to-host forward through pinned host buffers and device staging.
        packed: the automatic tiles with a packed copy read it too (scratch of
        the full copy, packed as the input arrives); DD_TILE_PACKED ranges
        always do."""
        per = _samples_per_elem(self.dtype)
        n = h_in.shape[1] * per if n_samp is None else int(n_samp)
        scratch = self._input_scratch(n, d_in_stage.device, 1 if packed else 0)
        check(self._lib.dd_run_host_scratch(
            self._h, h_in.data_ptr(), h_in.stride(0) * per, n, h_out.data_ptr(),
            d_in_stage.data_ptr(), d_out_stage.data_ptr(),
            None if scratch is None else scratch.data_ptr(),
            0 if scratch is None else scratch.numel(), _stream_ptr(stream)))
        if scratch is not None and stream is not None:
            scratch.record_stream(stream)

    def _check_input(self, x):
        import torch
        want = getattr(torch, _TORCH_DTYPE_NAMES[self.dtype])
        if x.dtype != want:
            raise TypeError(f"plan dtype {self.dtype} needs {want}, got {x.dtype}")
        if x.dim() != 2 or x.shape[0] != self.n_chan or x.stride(1) != 1:
            raise ValueError("x must be [n_chan][n_samp] with a contiguous time axis")
        if not x.is_cuda:
            raise ValueError("x must be a cuda tensor")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dd_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
