"""Python binding of the GB300 EPRL vertex library (C ABI in include/sf_eprl.h).

Argument marshalling only: every step of the computation runs in the CUDA kernels of
``libsf_eprl.so``. PyTorch supplies device memory and the current CUDA stream. There is no CPU
fallback: if the library is missing or no GPU is present the calls raise.

    import paper_2107_13952_gb300 as sf
    t = sf.sf_6j_table([sf.vertex((2,)*10, 1.2, 2)])
    sf.sf_boosters(t, (40.0, 40, 50))
    A, = sf.sf_vertex_amplitude(t)           # torch float64 tensor [i1][i2][i3][i4][i5] on cuda
"""
import ctypes
import os

from . import build as _build

_LIB = None
_LIB_PATH = _build.LIB

SF_OK, SF_ERR_ARG, SF_ERR_EMPTY, SF_ERR_OOM, SF_ERR_CUDA, SF_ERR_TIMEOUT, SF_ERR_NUMERIC, SF_ERR_LIMIT = \
    0, -1, -2, -3, -4, -5, -6, -7
SF_FP64, SF_MIXED, SF_MIXED_FF, SF_MIXED_TC, SF_MIXED_PX = 0, 1, 2, 3, 4
SF_TAB_6J, SF_TAB_6J_SLOTS, SF_TAB_D, SF_TAB_NODES = 1, 2, 3, 4

# names of every symbol declared in include/sf_eprl.h
EXPORTS = ("sf_version", "sf_last_error", "sf_intertwiner_ranges", "sf_output_ranges", "sf_num_shells", "sf_6j_table",
           "sf_6j_table_range",
           "sf_boosters", "sf_booster_shape", "sf_boosters_upload", "sf_boosters_download",
           "sf_vertex_amplitude", "sf_vertex_adjoint", "sf_table_size", "sf_table_copy", "sf_kernel_launches",
           "sf_last_kernel_ms", "sf_vertex_amplitude_noalloc", "sf_plan_create", "sf_plan_autotune",
           "sf_plan_run", "sf_plan_graph_launch", "sf_plan_sync", "sf_plan_info", "sf_plan_free",
           "sf_tables_free", "sf_check_dot2", "sf_contract_vectors", "sf_contract_vertices",
           "sf_delta3_amplitudes")


class SfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("sf error %d: %s" % (code, msg))
        self.code = code


class sf_vertex(ctypes.Structure):
    _fields_ = [("two_j", ctypes.c_int32 * 10), ("gamma", ctypes.c_double), ("dl", ctypes.c_int32),
                ("sub_first", ctypes.c_int32 * 5), ("sub_count", ctypes.c_int32 * 5)]


class sf_quad_rule(ctypes.Structure):
    _fields_ = [("r_max", ctypes.c_double), ("n_panels", ctypes.c_int32), ("order", ctypes.c_int32)]


class sf_tiling(ctypes.Structure):
    _fields_ = [("x_chunk", ctypes.c_int32), ("items_per_sm", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("i3_split", ctypes.c_int32)]


def vertex(two_j, gamma, dl, sub=None):
    """An ``sf_vertex``; ``sub`` (optional): five (first, count) pairs selecting a block of the
    intertwiner ranges for the output (count 0 = through the end of the range)."""
    v = sf_vertex()
    for i, t in enumerate(two_j):
        v.two_j[i] = int(t)
    v.gamma = float(gamma)
    v.dl = int(dl)
    if sub is not None:
        for e, (f, c) in enumerate(sub):
            v.sub_first[e] = int(f)
            v.sub_count[e] = int(c)
    return v


def _declare(lib):
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "sf_version": (ctypes.c_char_p, []),
        "sf_last_error": (ctypes.c_char_p, []),
        "sf_intertwiner_ranges": (ctypes.c_int, [ctypes.POINTER(sf_vertex), ctypes.POINTER(I32), ctypes.POINTER(I32)]),
        "sf_output_ranges": (ctypes.c_int, [ctypes.POINTER(sf_vertex), ctypes.POINTER(I32), ctypes.POINTER(I32)]),
        "sf_num_shells": (I64, [ctypes.POINTER(sf_vertex)]),
        "sf_6j_table": (ctypes.c_int, [ctypes.POINTER(sf_vertex), I32, ctypes.POINTER(P), P]),
        "sf_6j_table_range": (ctypes.c_int, [ctypes.POINTER(sf_vertex), I32, I64, I64, ctypes.POINTER(P), P]),
        "sf_boosters": (ctypes.c_int, [P, ctypes.POINTER(sf_quad_rule), P]),
        "sf_booster_shape": (ctypes.c_int, [P, I32, I32, ctypes.POINTER(I64)]),
        "sf_boosters_upload": (ctypes.c_int, [P, I32, I32, P, P]),
        "sf_boosters_download": (ctypes.c_int, [P, I32, I32, P, P]),
        "sf_vertex_amplitude": (ctypes.c_int, [P, ctypes.c_int, I64, I64, P, I64, ctypes.POINTER(P), P, P]),
        "sf_vertex_adjoint": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(P), P, ctypes.POINTER(P), ctypes.POINTER(P),
                                             P]),
        "sf_table_size": (I64, [P, I32, I32, I32]),
        "sf_table_copy": (ctypes.c_int, [P, I32, I32, I32, P, I64, P]),
        "sf_kernel_launches": (I64, []),
        "sf_last_kernel_ms": (D, [I32]),
        "sf_vertex_amplitude_noalloc": (ctypes.c_int, [P, I64, I64, ctypes.POINTER(P), P]),
        "sf_plan_create": (ctypes.c_int, [P, ctypes.c_int, I64, I64, ctypes.POINTER(sf_tiling), ctypes.POINTER(P),
                                          ctypes.POINTER(P)]),
        "sf_plan_autotune": (ctypes.c_int, [P, I64, ctypes.POINTER(sf_tiling), P]),
        "sf_plan_run": (ctypes.c_int, [P, P]),
        "sf_plan_graph_launch": (ctypes.c_int, [P, P]),
        "sf_plan_sync": (ctypes.c_int, [P, P]),
        "sf_plan_info": (ctypes.c_int, [P, ctypes.POINTER(sf_tiling), ctypes.POINTER(I64), ctypes.POINTER(I32),
                                        ctypes.POINTER(I64)]),
        "sf_plan_free": (None, [P]),
        "sf_tables_free": (None, [P]),
        "sf_check_dot2": (ctypes.c_int, [I32, I32, I32, P, P, P, P]),
        "sf_contract_vectors": (ctypes.c_int, [P, ctypes.POINTER(I32), I32, ctypes.POINTER(P), P, P]),
        "sf_contract_vertices": (ctypes.c_int, [P, P, I64, P, P]),
        "sf_delta3_amplitudes": (ctypes.c_int, [I32, ctypes.POINTER(P), ctypes.POINTER(I32), ctypes.POINTER(I32),
                                                ctypes.POINTER(I32), ctypes.POINTER(P), P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


def load(path=None):
    """Load (building first if needed) the in-tree CUDA library; raises if it cannot."""
    global _LIB
    if _LIB is not None:
        return _LIB
    p = path or _LIB_PATH
    if not os.path.exists(p):
        _build.build()
    lib = ctypes.CDLL(p)
    _declare(lib)
    _LIB = lib
    return lib


def _check(rc):
    if rc != SF_OK:
        raise SfError(rc, _LIB.sf_last_error().decode())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def intertwiner_ranges(two_j, gamma=1.2, dl=0):
    """(two_lo[5], dim[5]) of the intertwiners (host logic of the library, no device work)."""
    lib = load()
    v = vertex(two_j, gamma, dl)
    lo = (ctypes.c_int32 * 5)()
    dim = (ctypes.c_int32 * 5)()
    _check(lib.sf_intertwiner_ranges(ctypes.byref(v), lo, dim))
    return list(lo), list(dim)


def output_ranges(v):
    """(two_lo[5], dim[5]) of the tensors written for the ``sf_vertex`` v (its sub-range applied)."""
    lib = load()
    lo = (ctypes.c_int32 * 5)()
    dim = (ctypes.c_int32 * 5)()
    _check(lib.sf_output_ranges(ctypes.byref(v), lo, dim))
    return list(lo), list(dim)


def num_shells(two_j, gamma=1.2, dl=0):
    lib = load()
    v = vertex(two_j, gamma, dl)
    n = lib.sf_num_shells(ctypes.byref(v))
    if n < 0:
        _check(int(n))
    return int(n)


class Tables:
    """Owner of an ``sf_tables*`` (device tables of one or more vertices)."""

    def __init__(self, ptr, vertices):
        self.ptr = ptr
        self.vertices = list(vertices)

    def __del__(self):
        if getattr(self, "ptr", None) and _LIB is not None:
            _LIB.sf_tables_free(self.ptr)
            self.ptr = None

    def dims(self, vtx=0):
        """Output ranges (two_lo, dim) of vertex ``vtx`` (its sub-range applied)."""
        return output_ranges(self.vertices[vtx])


def sf_6j_table(vertices, stream=None, shell_range=None):
    """Tables of the vertices; with ``shell_range`` = (begin, end) only what those shells of every
    vertex read is built (``sf_6j_table_range``)."""
    lib = load()
    vs = list(vertices)
    arr = (sf_vertex * len(vs))(*vs)
    out = ctypes.c_void_p()
    if shell_range is None:
        _check(lib.sf_6j_table(arr, len(vs), ctypes.byref(out), _stream(stream)))
    else:
        _check(lib.sf_6j_table_range(arr, len(vs), int(shell_range[0]), int(shell_range[1]), ctypes.byref(out),
                                     _stream(stream)))
    return Tables(out, vs)


def sf_boosters(tables, rule=(40.0, 40, 50), stream=None):
    lib = load()
    q = sf_quad_rule(float(rule[0]), int(rule[1]), int(rule[2]))
    _check(lib.sf_boosters(tables.ptr, ctypes.byref(q), _stream(stream)))


def booster_shape(tables, vtx, edge):
    lib = load()
    sh = (ctypes.c_int64 * 3)()
    _check(lib.sf_booster_shape(tables.ptr, vtx, edge, sh))
    return tuple(sh)


def sf_boosters_download(tables, vtx, edge, stream=None):
    import torch
    lib = load()
    out = torch.zeros(booster_shape(tables, vtx, edge), dtype=torch.float64, device="cuda")
    _check(lib.sf_boosters_download(tables.ptr, vtx, edge, ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def sf_boosters_upload(tables, vtx, edge, B, stream=None):
    import torch
    lib = load()
    B = torch.as_tensor(B, dtype=torch.float64).contiguous()
    if tuple(B.shape) != booster_shape(tables, vtx, edge):
        raise ValueError("booster shape %s != %s" % (tuple(B.shape), booster_shape(tables, vtx, edge)))
    if B.device.type != "cuda":
        B = B.cuda()
    _check(lib.sf_boosters_upload(tables.ptr, vtx, edge, ctypes.c_void_p(B.data_ptr()), _stream(stream)))


def sf_vertex_amplitude(tables, precision=SF_FP64, shell_begin=0, shell_end=2 ** 63 - 1, shell_list=None,
                        out=None, stream=None, kappa=False):
    """Vertex tensors A[i1][i2][i3][i4][i5] (float64, cuda), one per vertex of ``tables``.

    precision: SF_FP64 (every step in FP64), SF_MIXED (booster contractions over k2, k3, k4 in
    FP32), SF_MIXED_FF (the same, with the {6j} contractions in compensated FP32 pairs),
    SF_MIXED_TC (the booster contractions FP32-class with k4 on the tensor cores in split BF16,
    the S3 contraction FP32, the x-sum FP64) or SF_MIXED_PX (the booster and S3 contractions in
    FP32 on the CUDA cores, the x-sum in compensated FP32 pairs); every mixed path stays within
    1e-6 (normwise, relative) of the FP64 result.
    With ``kappa`` True returns (tensors, sums) where sums[v] = sum_s ||C_s||_2 over the selected
    non-empty shells (one extra, unhoisted FP64 pass)."""
    import torch
    lib = load()
    outs = []
    for i, v in enumerate(tables.vertices):
        _, dim = output_ranges(v)
        if out is not None:
            o = out[i]
            assert o.dtype == torch.float64 and o.is_cuda and o.is_contiguous() and list(o.shape) == dim
        else:
            o = torch.empty(dim, dtype=torch.float64, device="cuda")
        outs.append(o)
    ptrs = (ctypes.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
    lp, nl = None, 0
    keep = None
    if shell_list is not None:
        keep = torch.as_tensor(shell_list, dtype=torch.int64).contiguous()
        if keep.device.type != "cuda":
            keep = keep.cuda()
        lp, nl = ctypes.c_void_p(keep.data_ptr()), int(keep.numel())
    kap = None
    if kappa:
        kap = torch.zeros(len(outs), dtype=torch.float64, device="cuda")
    _check(lib.sf_vertex_amplitude(tables.ptr, int(precision), int(shell_begin), int(shell_end), lp, nl, ptrs,
                                   ctypes.c_void_p(kap.data_ptr()) if kap is not None else None, _stream(stream)))
    if kappa:
        return outs, [float(v) for v in kap.cpu()]
    return outs


class Plan:
    """Owner of an ``sf_plan*``: one shell sum over a range of every vertex of ``tables``, set up
    once and run many times (``run``), optionally as a CUDA graph (``graph_launch``). Keeps the
    tables and the output tensors alive; ``outputs`` holds one float64 cuda tensor per vertex."""

    def __init__(self, tables, precision=SF_FP64, shell_begin=0, shell_end=2 ** 63 - 1, tiling=None):
        import torch
        lib = load()
        self.tables = tables
        self.outputs = []
        for v in tables.vertices:
            _, dim = output_ranges(v)
            self.outputs.append(torch.empty(dim, dtype=torch.float64, device="cuda"))
        ptrs = (ctypes.c_void_p * len(self.outputs))(*[o.data_ptr() for o in self.outputs])
        tl = sf_tiling(*(tuple(tiling or ()) + (0, 0, 0, 0))[:4])
        out = ctypes.c_void_p()
        _check(lib.sf_plan_create(tables.ptr, int(precision), int(shell_begin), int(shell_end), ctypes.byref(tl), ptrs,
                                  ctypes.byref(out)))
        self.ptr = out

    def autotune(self, sample_shells, stream=None):
        tl = sf_tiling()
        _check(load().sf_plan_autotune(self.ptr, int(sample_shells), ctypes.byref(tl), _stream(stream)))
        return (tl.x_chunk, tl.items_per_sm, tl.threads, tl.i3_split)

    def run(self, stream=None):
        _check(load().sf_plan_run(self.ptr, _stream(stream)))
        return self.outputs

    def graph_launch(self, stream=None):
        _check(load().sf_plan_graph_launch(self.ptr, _stream(stream)))
        return self.outputs

    def sync(self, stream=None):
        _check(load().sf_plan_sync(self.ptr, _stream(stream)))

    def info(self):
        tl, n, g, b = sf_tiling(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
        _check(load().sf_plan_info(self.ptr, ctypes.byref(tl), ctypes.byref(n), ctypes.byref(g), ctypes.byref(b)))
        return {"x_chunk": tl.x_chunk, "items_per_sm": tl.items_per_sm, "threads": tl.threads,
                "i3_split": tl.i3_split, "n_items": n.value, "grid": g.value, "scratch_bytes": b.value}

    def __del__(self):
        if getattr(self, "ptr", None) and _LIB is not None:
            _LIB.sf_plan_free(self.ptr)
            self.ptr = None


def kernel_launches():
    """Kernels launched by the library so far in this process."""
    return int(load().sf_kernel_launches())


def last_kernel_ms():
    """Device time (ms) of the last shell-sum kernel, from events on its stream."""
    return float(load().sf_last_kernel_ms(0))


def sf_vertex_amplitude_noalloc(tables, out, shell_begin=0, shell_end=2 ** 63 - 1, stream=None):
    """FP64 shell sum into caller-provided outputs without any device allocation by the library.

    For callers that must not allocate device memory while running (fixed memory pools, hosts that
    forbid allocation after start-up). ``out``: one preallocated cuda float64 tensor per vertex.
    The library's scratch is a fixed 32 MiB device array shared by all calls on a device, so calls
    that overlap on the GPU race; larger requests raise SfError(SF_ERR_LIMIT).
    """
    import torch
    lib = load()
    for i, v in enumerate(tables.vertices):
        _, dim = output_ranges(v)
        o = out[i]
        assert o.dtype == torch.float64 and o.is_cuda and o.is_contiguous() and list(o.shape) == dim
    ptrs = (ctypes.c_void_p * len(out))(*[o.data_ptr() for o in out])
    _check(lib.sf_vertex_amplitude_noalloc(tables.ptr, int(shell_begin), int(shell_end), ptrs, _stream(stream)))
    return out


def check_dot2(kind, a, b, stream=None):
    """Compensated-pair dot products on the device by the shell kernel's own steps (verification).

    kind 0: a float32 [n, len, 2] (hi, lo) pairs, b float32 [n, len]; kind 1: both [n, len, 2].
    Returns float32 [n, 2] (hi, lo) on the same device."""
    import torch
    lib = load()
    a = a.contiguous()
    b = b.contiguous()
    assert a.dtype == torch.float32 and b.dtype == torch.float32 and a.is_cuda and b.is_cuda
    n, ln = int(a.shape[0]), int(a.shape[1])
    out = torch.empty((n, 2), dtype=torch.float32, device=a.device)
    _check(lib.sf_check_dot2(int(kind), n, ln, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                             ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def _cplx(v, n):
    import torch
    v = torch.as_tensor(v).to(device="cuda", dtype=torch.complex128).contiguous()
    assert v.numel() == n, (v.numel(), n)
    return v


def contract_vectors(A, psis, stream=None):
    """Contract the vertex tensor A (cuda float64 [D1..D5]) with complex boundary vectors over its
    trailing len(psis) in {3, 4, 5} indices (psis[0] pairs with index 5 - len(psis)); returns the
    complex128 result on cuda: shape [D1, D2], [D1] or [] (Sec. 3, eq. vertex-contraction)."""
    import torch
    lib = load()
    assert A.dtype == torch.float64 and A.is_cuda and A.is_contiguous() and A.dim() == 5
    dims = list(A.shape)
    nv = len(psis)
    first = 5 - nv
    vs = [None] * first + [_cplx(p, dims[first + q]) for q, p in enumerate(psis)]
    ptrs = (ctypes.c_void_p * 5)(*[(v.data_ptr() if v is not None else None) for v in vs])
    shape = [[dims[0], dims[1]], [dims[0]], []][nv - 3]
    out = torch.empty(shape, dtype=torch.complex128, device="cuda")
    d = (ctypes.c_int32 * 5)(*dims)
    _check(lib.sf_contract_vectors(ctypes.c_void_p(A.data_ptr()), d, nv, ptrs, ctypes.c_void_p(out.data_ptr()),
                                   _stream(stream)))
    return out


def contract_vertices(A, B, stream=None):
    """sum_i A[i] B[i] of two vertex tensors of equal shape (cuda float64); a cuda float64 scalar."""
    import torch
    lib = load()
    assert A.shape == B.shape and A.dtype == B.dtype == torch.float64 and A.is_contiguous() and B.is_contiguous()
    out = torch.empty((), dtype=torch.float64, device="cuda")
    _check(lib.sf_contract_vertices(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()), A.numel(),
                                    ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def delta3_amplitudes(tensors, two_x, two_klo, psis, stream=None):
    """Delta_3 amplitudes per internal spin and their sum (Sec. 5): ``tensors`` the vertex tensors
    A_x (cuda float64, one per x), ``two_x``/``two_klo`` their doubled internal spins and lowest
    internal intertwiners, ``psis`` nine boundary vectors (three per vertex, on i3, i4, i5).
    Returns (amps [n_x] complex128, total complex128 scalar), both on cuda."""
    import torch
    lib = load()
    n = len(tensors)
    dims = []
    for A in tensors:
        assert A.dtype == torch.float64 and A.is_cuda and A.is_contiguous() and A.dim() == 5
        dims += list(A.shape)
    bd = list(tensors[0].shape[2:]) * 3
    vs = [_cplx(p, bd[q]) for q, p in enumerate(psis)]
    amps = torch.empty(n, dtype=torch.complex128, device="cuda")
    total = torch.empty((), dtype=torch.complex128, device="cuda")
    _check(lib.sf_delta3_amplitudes(n, (ctypes.c_void_p * n)(*[A.data_ptr() for A in tensors]),
                                    (ctypes.c_int32 * (5 * n))(*dims), (ctypes.c_int32 * n)(*two_x),
                                    (ctypes.c_int32 * n)(*two_klo), (ctypes.c_void_p * 9)(*[v.data_ptr() for v in vs]),
                                    ctypes.c_void_p(amps.data_ptr()), ctypes.c_void_p(total.data_ptr()),
                                    _stream(stream)))
    return amps, total


def table_copy(tables, vtx, kind, index, stream=None):
    """Copy an internal table to a CPU torch tensor (verification only)."""
    import torch
    lib = load()
    n = lib.sf_table_size(tables.ptr, vtx, kind, index)
    if n < 0:
        _check(int(n))
    if kind == SF_TAB_6J_SLOTS:
        out = torch.zeros(max(1, n // 8), dtype=torch.int64)
    else:
        out = torch.zeros(max(1, n // 8), dtype=torch.float64)
    _check(lib.sf_table_copy(tables.ptr, vtx, kind, index, ctypes.c_void_p(out.data_ptr()), int(n), _stream(stream)))
    if kind == SF_TAB_6J_SLOTS:
        return out.view(-1, 8)
    if kind == SF_TAB_D:
        return torch.view_as_complex(out.view(-1, 2))
    return out


def sf_vertex_adjoint(tables, psis, want_grads=True, precision=SF_FP64, stream=None):
    """(a, [d a/d psi_e], [d a/d B_e]) for complex boundary vectors psis (cuda complex128); with
    ``want_grads`` False only a is computed (the gradient lists are empty)."""
    import torch
    lib = load()
    psis = [torch.as_tensor(p, dtype=torch.complex128).contiguous().cuda() for p in psis]
    a = torch.zeros(1, dtype=torch.complex128, device="cuda")
    pp = (ctypes.c_void_p * 5)(*[p.data_ptr() for p in psis])
    gp, gb = None, None
    gps, gbs = [], []
    if want_grads:
        gps = [torch.zeros_like(p) for p in psis]
        gbs = [torch.zeros(booster_shape(tables, 0, e), dtype=torch.complex128, device="cuda") for e in (2, 3, 4, 5)]
        gp = (ctypes.c_void_p * 5)(*[g.data_ptr() for g in gps])
        gb = (ctypes.c_void_p * 4)(*[g.data_ptr() for g in gbs])
    _check(lib.sf_vertex_adjoint(tables.ptr, int(precision), pp, ctypes.c_void_p(a.data_ptr()), gp, gb,
                                 _stream(stream)))
    return a[0], gps, gbs


def vjp_from_holomorphic(grad_out, G, real_input):
    """Backward rule for a function holomorphic in its complex inputs and real-linear in its real
    inputs, given its holomorphic derivative G = d out / d input: PyTorch passes grad_out =
    dL/d conj(out) and expects dL/d conj(input) = grad_out * conj(G) for complex inputs, and the
    real part of that for real inputs."""
    g = grad_out * G.conj()
    return g.real if real_input else g


def _contraction_function():
    import torch

    class EPRLContraction(torch.autograd.Function):
        """a = sum_i A[i] prod_e psi_e[i_e] for one vertex, differentiable in the five complex
        boundary vectors and the four real booster tensors (forward and backward both run in the
        library's adjoint kernels, which recompute every shell's {15j} ring)."""

        @staticmethod
        def forward(ctx, tables, psi1, psi2, psi3, psi4, psi5, B2, B3, B4, B5):
            for e, B in zip((2, 3, 4, 5), (B2, B3, B4, B5)):
                sf_boosters_upload(tables, 0, e, B.detach())
            psis = [p.detach() for p in (psi1, psi2, psi3, psi4, psi5)]
            # the gradients come from the same kernels as a; skip them when nothing needs them
            need = any(ctx.needs_input_grad[1:])
            a, gpsi, gB = sf_vertex_adjoint(tables, psis, want_grads=need)
            ctx.has_grads = need
            if need:
                ctx.save_for_backward(*gpsi, *gB)
            return a.clone()

        @staticmethod
        def backward(ctx, grad_a):
            saved = ctx.saved_tensors
            gpsi = [vjp_from_holomorphic(grad_a, g, False) for g in saved[:5]]
            gB = [vjp_from_holomorphic(grad_a, g, True) for g in saved[5:]]
            return (None, *gpsi, *gB)

    return EPRLContraction


_EPRL_FN = None


def eprl_contraction(tables, psis, boosters):
    """Differentiable boundary-contracted amplitude (torch.autograd.Function over the C ABI).

    psis: five complex128 cuda tensors (boundary intertwiner vectors); boosters: four float64 cuda
    tensors shaped like ``booster_shape(tables, 0, e)`` for e = 2..5.
    """
    global _EPRL_FN
    if _EPRL_FN is None:
        _EPRL_FN = _contraction_function()
    return _EPRL_FN.apply(tables, *psis, *boosters)
