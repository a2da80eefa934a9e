"""Thin ctypes binding of libdonof (include/donof.h): same names, argument marshalling only.

Every step of a build runs in the library's CUDA kernels.  PyTorch provides device
memory and the current CUDA stream; nothing here computes on the host.  The library
must have been built (``paper_2004_06142_gb300.build.build()``); loading fails loudly
otherwise.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdonof.so")

PNOF5, PNOF7, PNOF7S = 5, 7, 8
B_DENSE, B_PACKED = 0, 1
FP64, MIXED = 0, 1

STATUS = {
    0: "ok", -1: "invalid argument", -2: "pair_map violates the subspace layout",
    -3: "non-finite input or result", -4: "workspace too small or misaligned",
    -5: "CUDA call failed", -6: "device wait limit exceeded", -7: "unsupported problem size",
    -8: "donof_prepare_B not called for this workspace and B",
}


class DonofError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, 'unknown status')} ({code})")
        self.code = code


BATCH_BACKWARD, BATCH_GRAPH, BATCH_STREAMS = 1, 2, 4
ERR_WORKSPACE = -4


def alloc_workspace(nbytes: int, device) -> torch.Tensor:
    """Device workspace of nbytes.  An allocation failure is reported as DonofError with
    the workspace status; DONOF_INJECT_ALLOC_FAILURE=1 in the environment makes every such
    allocation fail that way (host-side fault injection, no device involved)."""
    if os.environ.get("DONOF_INJECT_ALLOC_FAILURE") == "1":
        raise DonofError(ERR_WORKSPACE, f"workspace allocation of {nbytes} bytes (injected failure)")
    try:
        return torch.empty(nbytes, dtype=torch.uint8, device=device)
    except (RuntimeError, MemoryError) as e:  # torch.OutOfMemoryError derives from RuntimeError
        raise DonofError(ERR_WORKSPACE, f"workspace allocation of {nbytes} bytes: {e}") from e


class donof_instance(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("h", "B", "C", "gamma", "pair_map", "E", "lam",
                                              "dE_dgamma", "dE_dC")]


class donof_opt_params(ctypes.Structure):
    _fields_ = [("max_outer", ctypes.c_int32), ("max_inner", ctypes.c_int32),
                ("diis_depth", ctypes.c_int32), ("occ_max_iter", ctypes.c_int32),
                ("zeta", ctypes.c_double), ("delta", ctypes.c_double),
                ("eps_energy", ctypes.c_double), ("occ_gtol", ctypes.c_double)]


class donof_opt_result(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("max_asym", ctypes.c_double),
                ("outer", ctypes.c_int32), ("inner", ctypes.c_int32), ("builds", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("energies_recorded", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class donof_problem(ctypes.Structure):
    _fields_ = [("nbf", ctypes.c_int32), ("naux", ctypes.c_int32), ("npair", ctypes.c_int32),
                ("ncwo", ctypes.c_int32), ("functional", ctypes.c_int32),
                ("b_layout", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("nsingle", ctypes.c_int32), ("x_budget_bytes", ctypes.c_uint64)]


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libdonof.so is not built ({LIB_PATH}); run "
                               "paper_2004_06142_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER(donof_problem)
        vp, sz = ctypes.c_void_p, ctypes.c_size_t
        L.donof_workspace_size.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
        L.donof_prepare_B.argtypes = [P, vp, vp, sz, vp]
        L.donof_energy_lagrangian.argtypes = [P, vp, vp, vp, vp, vp, vp, sz, vp, vp, vp, vp]
        L.donof_energy_backward.argtypes = [P, vp, vp, sz, vp, vp, vp]
        L.donof_get_jk.argtypes = [P, vp, sz, vp, vp, vp]
        L.donof_partial_size.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
        L.donof_energy_lagrangian_partial.argtypes = [P, vp, vp, vp, vp, vp, vp, sz, vp, vp]
        L.donof_energy_lagrangian_finish.argtypes = [P, vp, vp, vp, vp, vp, vp, sz, vp, vp, vp, vp]
        L.donof_read_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), vp]
        L.donof_status_string.argtypes = [ctypes.c_int]
        L.donof_status_string.restype = ctypes.c_char_p
        L.donof_energy_lagrangian_noalloc.argtypes = [P, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.donof_noalloc_read_status.argtypes = [ctypes.POINTER(ctypes.c_int32), vp]
        PI = ctypes.POINTER(donof_instance)
        L.donof_batched_workspace_size.argtypes = [ctypes.c_int32, P, ctypes.POINTER(ctypes.c_size_t)]
        L.donof_prepare_B_batched.argtypes = [ctypes.c_int32, P, PI, vp, sz, vp]
        L.donof_energy_lagrangian_batched.argtypes = [ctypes.c_int32, P, PI, vp, sz, ctypes.c_int32, vp]
        L.donof_orbital_update_workspace_size.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]
        L.donof_orbital_update.argtypes = [ctypes.c_int32, vp, vp, vp, vp, sz, vp, vp, vp]
        L.donof_host_staging_size.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
        L.donof_energy_lagrangian_host.argtypes = [P, vp, vp, vp, vp, vp, vp, sz, vp, sz, vp, vp,
                                                   vp, vp, vp]
        L.donof_eigh_workspace_size.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]
        L.donof_eigh.argtypes = [ctypes.c_int32, vp, vp, vp, vp, sz, vp]
        L.donof_eigh_read_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), vp]
        L.donof_autotune.argtypes = [P, vp, vp, vp, vp, vp, vp, sz, vp]
        L.donof_optimize_occupations.argtypes = [P, vp, vp, vp, sz, ctypes.c_int32,
                                                 ctypes.c_double, vp, vp, vp]
        L.donof_optimize_workspace_size.argtypes = [P, ctypes.c_int32,
                                                    ctypes.POINTER(ctypes.c_size_t)]
        L.donof_optimize.argtypes = [P, ctypes.POINTER(donof_opt_params), vp, vp, vp, vp, vp, vp,
                                     ctypes.c_int32, vp, sz, vp, sz,
                                     ctypes.POINTER(donof_opt_result), vp, ctypes.c_int32, vp]
        L.donof_nofmp2_static.argtypes = [P, vp, vp, sz, vp, vp, vp]
        L.donof_profile_enable.argtypes = [ctypes.c_int32]
        L.donof_profile_read.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int32)]
        L.donof_launch_count.argtypes = []
        L.donof_launch_count.restype = ctypes.c_int64
        for f in ("donof_workspace_size", "donof_prepare_B", "donof_energy_lagrangian",
                  "donof_energy_backward", "donof_get_jk", "donof_read_status",
                  "donof_profile_enable", "donof_profile_read", "donof_energy_lagrangian_noalloc",
                  "donof_noalloc_read_status", "donof_partial_size",
                  "donof_energy_lagrangian_partial", "donof_energy_lagrangian_finish",
                  "donof_batched_workspace_size", "donof_prepare_B_batched",
                  "donof_energy_lagrangian_batched", "donof_orbital_update_workspace_size",
                  "donof_orbital_update", "donof_eigh_workspace_size", "donof_eigh",
                  "donof_host_staging_size", "donof_energy_lagrangian_host",
                  "donof_eigh_read_status", "donof_autotune", "donof_optimize_occupations",
                  "donof_optimize_workspace_size", "donof_optimize", "donof_nofmp2_static"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def make_problem(nbf, naux, npair, ncwo, functional=PNOF7, b_layout=B_DENSE, precision=FP64,
                 x_budget_bytes=0, nsingle=0) -> donof_problem:
    return donof_problem(nbf, naux, npair, ncwo, functional, b_layout, precision, nsingle,
                         x_budget_bytes)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(rc: int, where: str):
    if rc != 0:
        raise DonofError(rc, where)


def donof_workspace_size(prob: donof_problem) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().donof_workspace_size(ctypes.byref(prob), ctypes.byref(n)), "donof_workspace_size")
    return n.value


def donof_prepare_B(prob, B, ws, stream=None):
    _check(lib().donof_prepare_B(ctypes.byref(prob), _ptr(B), _ptr(ws), ws.numel(), _stream(stream)),
           "donof_prepare_B")


def donof_energy_lagrangian(prob, h, B, C, gamma, pair_map, ws, E, lam=None, dE_dgamma=None,
                            stream=None):
    _check(lib().donof_energy_lagrangian(ctypes.byref(prob), _ptr(h), _ptr(B), _ptr(C), _ptr(gamma),
                                         _ptr(pair_map), _ptr(ws), ws.numel(), _ptr(E), _ptr(lam),
                                         _ptr(dE_dgamma), _stream(stream)),
           "donof_energy_lagrangian")


def donof_partial_size(prob: donof_problem) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().donof_partial_size(ctypes.byref(prob), ctypes.byref(n)), "donof_partial_size")
    return n.value


def donof_energy_lagrangian_partial(prob, h, B, C, gamma, pair_map, ws, partial, stream=None):
    _check(lib().donof_energy_lagrangian_partial(ctypes.byref(prob), _ptr(h), _ptr(B), _ptr(C),
                                                 _ptr(gamma), _ptr(pair_map), _ptr(ws),
                                                 ws.numel(), _ptr(partial), _stream(stream)),
           "donof_energy_lagrangian_partial")


def donof_energy_lagrangian_finish(prob, h, C, gamma, pair_map, partial, ws, E, lam=None,
                                   dE_dgamma=None, stream=None):
    _check(lib().donof_energy_lagrangian_finish(ctypes.byref(prob), _ptr(h), _ptr(C), _ptr(gamma),
                                                _ptr(pair_map), _ptr(partial), _ptr(ws),
                                                ws.numel(), _ptr(E), _ptr(lam), _ptr(dE_dgamma),
                                                _stream(stream)),
           "donof_energy_lagrangian_finish")


def shard_range(naux: int, rank: int, world: int):
    """The auxiliary slices [P0, P1) of shard `rank` out of `world`: contiguous, sizes
    differing by at most one."""
    return naux * rank // world, naux * (rank + 1) // world


def exchange_partial(partial: torch.Tensor, group=None) -> torch.Tensor:
    """The one exchange of a sharded build: every rank's partial sums (J, K, two-electron G)
    replaced in place by their sum over the ranks of the process group (an all-reduce; NCCL
    for device tensors, gloo for host tensors).  Returns `partial`."""
    import torch.distributed as tdist
    if tdist.is_available() and tdist.is_initialized() and tdist.get_world_size(group) > 1:
        tdist.all_reduce(partial, op=tdist.ReduceOp.SUM, group=group)
    return partial


def donof_energy_backward(prob, Ebar, ws, dE_dC=None, dE_dgamma=None, stream=None):
    _check(lib().donof_energy_backward(ctypes.byref(prob), _ptr(Ebar), _ptr(ws), ws.numel(),
                                       _ptr(dE_dC), _ptr(dE_dgamma), _stream(stream)),
           "donof_energy_backward")


def donof_energy_lagrangian_noalloc(prob, h, B, C, gamma, pair_map, E, lam=None, dE_dgamma=None,
                                    dE_dC=None, stream=None):
    """One build (and optionally dE/dC) using the library's fixed device scratch: no device
    memory is allocated.  Small problems only (see include/donof.h)."""
    _check(lib().donof_energy_lagrangian_noalloc(ctypes.byref(prob), _ptr(h), _ptr(B), _ptr(C),
                                                 _ptr(gamma), _ptr(pair_map), _ptr(E), _ptr(lam),
                                                 _ptr(dE_dgamma), _ptr(dE_dC), _stream(stream)),
           "donof_energy_lagrangian_noalloc")


def donof_noalloc_read_status(stream=None) -> int:
    """Device status of the last allocation-free build on the current device (then cleared)."""
    st = ctypes.c_int32(0)
    _check(lib().donof_noalloc_read_status(ctypes.byref(st), _stream(stream)),
           "donof_noalloc_read_status")
    return st.value


def donof_orbital_update(lam, Fdiag, C, C_new, eps, ws=None, stream=None):
    """F of Eq. Fockian from lambda and a given diagonal, its eigendecomposition, C_new = C V
    reorthonormalised (all on the device).  Returns the workspace used."""
    n = C.shape[0]
    if ws is None:
        nb = ctypes.c_size_t(0)
        _check(lib().donof_orbital_update_workspace_size(n, ctypes.byref(nb)),
               "donof_orbital_update_workspace_size")
        ws = alloc_workspace(nb.value, C.device)
    _check(lib().donof_orbital_update(n, _ptr(lam), _ptr(Fdiag), _ptr(C), _ptr(ws), ws.numel(),
                                      _ptr(C_new), _ptr(eps), _stream(stream)),
           "donof_orbital_update")
    return ws


def _hptr(t):
    if t is None:
        return None
    if t.is_cuda or not t.is_contiguous():
        raise ValueError("contiguous host tensor expected")
    return ctypes.c_void_p(t.data_ptr())


def donof_host_staging_size(prob) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().donof_host_staging_size(ctypes.byref(prob), ctypes.byref(n)),
           "donof_host_staging_size")
    return n.value


def donof_energy_lagrangian_host(prob, h, B, C_host, gamma_host, pair_map, ws, staging, E_host,
                                 lam_host=None, dEdg_host=None, dEdC_host=None, stream=None):
    """One build (and its adjoint when dEdC_host is given) from host C and gamma into host
    outputs; h, B, pair_map, ws and staging are device tensors.  Returns after the stream is
    idle; raises DonofError with the build's device-side status when it is not DONOF_OK."""
    _check(lib().donof_energy_lagrangian_host(
        ctypes.byref(prob), _ptr(h), _ptr(B), _hptr(C_host), _hptr(gamma_host), _ptr(pair_map),
        _ptr(ws), ws.numel(), _ptr(staging), staging.numel(), _hptr(E_host), _hptr(lam_host),
        _hptr(dEdg_host), _hptr(dEdC_host), _stream(stream)), "donof_energy_lagrangian_host")


def donof_eigh(A, V, w, ws=None, stream=None):
    """A = V diag(w) V^T in double on the device (w ascending, column j of V eigenvector j);
    V may be A.  Returns the workspace used."""
    n = A.shape[0]
    if ws is None:
        nb = ctypes.c_size_t(0)
        _check(lib().donof_eigh_workspace_size(n, ctypes.byref(nb)), "donof_eigh_workspace_size")
        ws = alloc_workspace(nb.value, A.device)
    _check(lib().donof_eigh(n, _ptr(A), _ptr(V), _ptr(w), _ptr(ws), ws.numel(), _stream(stream)),
           "donof_eigh")
    return ws


def donof_eigh_read_status(ws, stream=None):
    """Device-side status of the last donof_eigh on ``ws`` (waits for the stream)."""
    st = ctypes.c_int32(0)
    _check(lib().donof_eigh_read_status(_ptr(ws), ctypes.byref(st), _stream(stream)),
           "donof_eigh_read_status")
    return st.value


def donof_optimize_occupations(prob, pair_map, gamma, ws, max_iter=500, gtol=1e-9, E=None,
                               iters=None, stream=None):
    """L-BFGS over gamma at the orbitals of the last build on ``ws`` (gamma updated in place)."""
    _check(lib().donof_optimize_occupations(ctypes.byref(prob), _ptr(pair_map), _ptr(gamma),
                                            _ptr(ws), ws.numel(), int(max_iter), float(gtol),
                                            _ptr(E), _ptr(iters), _stream(stream)),
           "donof_optimize_occupations")


def donof_nofmp2_static(prob, pair_map, ws, E_hf, E_sta, stream=None):
    _check(lib().donof_nofmp2_static(ctypes.byref(prob), _ptr(pair_map), _ptr(ws), ws.numel(),
                                     _ptr(E_hf), _ptr(E_sta), _stream(stream)),
           "donof_nofmp2_static")


def donof_get_jk(prob, ws, J=None, K=None, stream=None):
    _check(lib().donof_get_jk(ctypes.byref(prob), _ptr(ws), ws.numel(), _ptr(J), _ptr(K),
                              _stream(stream)), "donof_get_jk")


def donof_read_status(ws, stream=None) -> int:
    st = ctypes.c_int32(0)
    _check(lib().donof_read_status(_ptr(ws), ctypes.byref(st), _stream(stream)), "donof_read_status")
    return st.value


PHASES = ["prep", "half_transform", "mo_3index", "jk_y", "g_build", "energy_lambda",
          "backward", "prepare_B", "orbital_update", "occ_opt", "orbital_step"]


def donof_profile_enable(enable: bool):
    _check(lib().donof_profile_enable(1 if enable else 0), "donof_profile_enable")


def donof_profile_read(phase: int):
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int32(0)
    _check(lib().donof_profile_read(phase, ctypes.byref(ms), ctypes.byref(n)), "donof_profile_read")
    return ms.value, n.value


def donof_launch_count() -> int:
    return int(lib().donof_launch_count())


def donof_status_string(code: int) -> str:
    return lib().donof_status_string(code).decode()


# ---------------------------------------------------------------------------
class Builder:
    """Owns a workspace for one problem and one prepared B (device tensors)."""

    def __init__(self, nbf, naux, npair, ncwo, functional=PNOF7, b_layout=B_DENSE,
                 precision=FP64, x_budget_bytes=0, device="cuda", nsingle=0):
        self.prob = make_problem(nbf, naux, npair, ncwo, functional, b_layout, precision,
                                 x_budget_bytes, nsingle)
        self.nbf, self.naux, self.npair, self.ncwo = nbf, naux, npair, ncwo
        self.nsingle = nsingle
        self.nact = npair * (1 + ncwo) + nsingle
        self.ngamma = npair * ncwo
        self.device = torch.device(device)
        self.ws = alloc_workspace(donof_workspace_size(self.prob), self.device)
        self.B = None

    def prepare(self, B: torch.Tensor):
        self.B = B
        donof_prepare_B(self.prob, B, self.ws)

    def autotune(self, h, C, gamma, pair_map):
        """Pick the tensor-core tile widths for this shape by timing builds (mixed only)."""
        _check(lib().donof_autotune(ctypes.byref(self.prob), _ptr(h), _ptr(self.B), _ptr(C),
                                    _ptr(gamma), _ptr(pair_map), _ptr(self.ws), self.ws.numel(),
                                    _stream(None)), "donof_autotune")

    def forward(self, h, C, gamma, pair_map, want_lam=True):
        dev, f64 = self.device, torch.float64
        E = torch.empty(1, dtype=f64, device=dev)
        lam = torch.empty(self.nbf, self.nbf, dtype=f64, device=dev) if want_lam else None
        dEdg = torch.empty(self.ngamma, dtype=f64, device=dev)
        donof_energy_lagrangian(self.prob, h, self.B, C, gamma, pair_map, self.ws, E, lam, dEdg)
        return E, lam, dEdg

    def forward_partial(self, h, C, gamma, pair_map, partial=None):
        """This shard's partial sums (J, K, two-electron G) over the slices of the prepared B,
        as one flat double tensor of donof_partial_size elements."""
        if partial is None:
            partial = torch.empty(donof_partial_size(self.prob), dtype=torch.float64,
                                  device=self.device)
        donof_energy_lagrangian_partial(self.prob, h, self.B, C, gamma, pair_map, self.ws, partial)
        return partial

    def finish(self, h, C, gamma, pair_map, partial, want_lam=True):
        """E, lambda, dE/dgamma from the partial sums of every shard, summed."""
        dev, f64 = self.device, torch.float64
        E = torch.empty(1, dtype=f64, device=dev)
        lam = torch.empty(self.nbf, self.nbf, dtype=f64, device=dev) if want_lam else None
        dEdg = torch.empty(self.ngamma, dtype=f64, device=dev)
        donof_energy_lagrangian_finish(self.prob, h, C, gamma, pair_map, partial, self.ws, E, lam,
                                       dEdg)
        return E, lam, dEdg

    def forward_sharded(self, h, C, gamma, pair_map, group=None, want_lam=True):
        """One build of a problem whose auxiliary index is sharded over the ranks of a
        torch.distributed process group (this Builder holds this rank's slices): the shard's
        partial sums, their all-reduce (sum) over the group, then E, lambda, dE/dgamma on every
        rank."""
        partial = exchange_partial(self.forward_partial(h, C, gamma, pair_map), group)
        return self.finish(h, C, gamma, pair_map, partial, want_lam)

    def backward(self, Ebar):
        dev, f64 = self.device, torch.float64
        dC = torch.empty(self.nbf, self.nbf, dtype=f64, device=dev)
        dg = torch.empty(self.ngamma, dtype=f64, device=dev)
        donof_energy_backward(self.prob, Ebar, self.ws, dC, dg)
        return dC, dg

    def optimize_occupations(self, gamma, pair_map, max_iter=500, gtol=1e-9):
        """Optimal gamma (in place), its energy and the iterations taken, at the orbitals of
        the last forward()."""
        E = torch.empty(1, dtype=torch.float64, device=self.device)
        it = torch.zeros(1, dtype=torch.int32, device=self.device)
        donof_optimize_occupations(self.prob, pair_map, gamma, self.ws, max_iter, gtol, E, it)
        return E, it

    def nofmp2_static(self, pair_map):
        """The HF-like energy and the static correlation energy of NOF-MP2 (Eqs. HFL, Esta)
        at the orbitals and occupations of the last forward(); device scalars."""
        E_hf = torch.empty(1, dtype=torch.float64, device=self.device)
        E_sta = torch.empty(1, dtype=torch.float64, device=self.device)
        donof_nofmp2_static(self.prob, pair_map, self.ws, E_hf, E_sta)
        return E_hf, E_sta

    def optimize(self, h, C, gamma, pair_map, Fdiag=None, max_outer=50, max_inner=10,
                 diis_depth=6, zeta=1.0, delta=1e-6, eps_energy=1e-10, occ_max_iter=500,
                 occ_gtol=1e-10, max_energies=4096):
        """The optimisation procedure (donof_optimize): C, gamma and the diagonal (returned)
        are updated in place; with Fdiag None the initial diagonal comes from the
        symmetrised lambda.  Returns (result dict, energies of the orbital iterations)."""
        prm = donof_opt_params(max_outer, max_inner, diis_depth, occ_max_iter, zeta, delta,
                               eps_energy, occ_gtol)
        nb = ctypes.c_size_t(0)
        _check(lib().donof_optimize_workspace_size(ctypes.byref(self.prob), diis_depth,
                                                   ctypes.byref(nb)),
               "donof_optimize_workspace_size")
        ows = alloc_workspace(nb.value, self.device)
        init = Fdiag is None
        if init:
            Fdiag = torch.zeros(self.nbf, dtype=torch.float64, device=self.device)
        res = donof_opt_result()
        energies = (ctypes.c_double * max(max_energies, 1))()
        _check(lib().donof_optimize(ctypes.byref(self.prob), ctypes.byref(prm), _ptr(h),
                                    _ptr(self.B), _ptr(C), _ptr(gamma), _ptr(pair_map),
                                    _ptr(Fdiag), 1 if init else 0, _ptr(self.ws),
                                    self.ws.numel(), _ptr(ows), ows.numel(), ctypes.byref(res),
                                    energies, max_energies, _stream(None)), "donof_optimize")
        out = dict(E=res.E, max_asym=res.max_asym, outer=res.outer, inner=res.inner,
                   builds=res.builds, converged=bool(res.converged), Fdiag=Fdiag)
        n = min(res.energies_recorded, max_energies)
        return out, [energies[i] for i in range(n)]

    def jk(self):
        J = torch.empty(self.nact, self.nact, dtype=torch.float64, device=self.device)
        K = torch.empty_like(J)
        donof_get_jk(self.prob, self.ws, J, K)
        return J, K

    def status(self) -> int:
        return donof_read_status(self.ws)


def donof_batched_workspace_size(probs) -> int:
    arr = (donof_problem * len(probs))(*probs)
    n = ctypes.c_size_t(0)
    _check(lib().donof_batched_workspace_size(len(probs), arr, ctypes.byref(n)),
           "donof_batched_workspace_size")
    return n.value


class Batch:
    """Many independent instances in one call (library-owned streams, optional CUDA graph).

    ``instances`` is a list of dicts of device tensors: h, B, C, gamma, pair_map and the
    outputs E, lam, dE_dgamma, dE_dC (outputs may be missing)."""

    def __init__(self, probs, instances, device="cuda"):
        self.n = len(probs)
        self.probs = (donof_problem * self.n)(*probs)
        self.tensors = instances  # keeps the tensors alive
        rows = []
        for x in instances:
            rows.append(donof_instance(*[(x[k].data_ptr() if x.get(k) is not None else None)
                                         for k in ("h", "B", "C", "gamma", "pair_map", "E", "lam",
                                                   "dE_dgamma", "dE_dC")]))
        self.inst = (donof_instance * self.n)(*rows)
        self.ws = alloc_workspace(donof_batched_workspace_size(probs), device)

    def prepare(self, stream=None):
        _check(lib().donof_prepare_B_batched(self.n, self.probs, self.inst, _ptr(self.ws),
                                             self.ws.numel(), _stream(stream)),
               "donof_prepare_B_batched")

    def run(self, flags=BATCH_BACKWARD, stream=None):
        _check(lib().donof_energy_lagrangian_batched(self.n, self.probs, self.inst, _ptr(self.ws),
                                                     self.ws.numel(), flags, _stream(stream)),
               "donof_energy_lagrangian_batched")

    def status(self) -> int:
        """The batch's status word (wait limits of the grouped launches), then cleared."""
        return donof_read_status(self.ws)


class DonofEnergy(torch.autograd.Function):
    """E(C, gamma) with the library's adjoint: dE/dC = 4 Ebar G, dE/dgamma = Ebar dE/dgamma.
    lambda is returned as a non-differentiable output."""

    @staticmethod
    def forward(ctx, C, gamma, builder: Builder, h, pair_map):
        E, lam, _ = builder.forward(h, C.contiguous(), gamma.contiguous(), pair_map)
        ctx.builder = builder
        ctx.mark_non_differentiable(lam)
        return E.reshape(()), lam

    @staticmethod
    def backward(ctx, gE, glam):
        Ebar = gE.reshape(1).to(torch.float64).contiguous()
        dC, dg = ctx.builder.backward(Ebar)
        return dC, dg, None, None, None


def energy(C, gamma, builder: Builder, h, pair_map):
    """Differentiable energy (and lambda) of one build."""
    return DonofEnergy.apply(C, gamma, builder, h, pair_map)
