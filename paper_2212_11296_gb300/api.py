"""Python face of the C ABI: torch tensors and streams in, library calls out."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib

REUSE = _lib.REUSE
BF16 = _lib.BF16
INCREMENTAL = _lib.INCREMENTAL
BF16_SPLIT = _lib.BF16_SPLIT

_LIB = None


def lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = _lib.load()
    return _LIB


class VQNQSError(RuntimeError):
    pass


def _stream_ptr(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _check_dev(t: torch.Tensor, dtype, name):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")


class VQNQS:
    """One model on one lattice: vqnqs_create(L, periodic, J, layers, d_model, heads, K, weights), or
    vqnqs_create_arch(..., K, vq_heads, half_block, token_group, weights) for quantizers with vq_heads
    heads of K codes each, the final attention-only half-block and/or tokens of token_group spins."""

    def __init__(self, L: int, periodic: bool, J: float, layers: int, d_model: int, heads: int, K: int,
                 weights: np.ndarray, vq_heads: int = 1, half_block: bool = False, token_group: int = 1):
        self.L, self.N = L, L * L
        self.periodic, self.J = bool(periodic), float(J)
        self.layers, self.d, self.heads, self.K = layers, d_model, heads, K
        self.vq_heads, self.half_block, self.token_group = int(vq_heads), bool(half_block), int(token_group)
        w = np.ascontiguousarray(weights, dtype=np.float32)
        n = lib().vqnqs_num_params_arch(self.N, layers, d_model, K, int(self.half_block), self.token_group)
        if w.size != n:
            raise ValueError(f"weight blob has {w.size} floats, layout needs {n}")
        h = ctypes.c_void_p()
        if self.vq_heads == 1 and not self.half_block and self.token_group == 1:
            rc = lib().vqnqs_create(L, int(periodic), float(J), layers, d_model, heads, K,
                                    w.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h))
        else:
            rc = lib().vqnqs_create_arch(L, int(periodic), float(J), layers, d_model, heads, K, self.vq_heads,
                                         int(self.half_block), self.token_group, w.ctypes.data_as(ctypes.c_void_p),
                                         ctypes.byref(h))
        if rc != 0:
            raise VQNQSError(f"vqnqs_create failed: {_lib.STATUS_NAMES.get(rc, rc)}")
        self._h = h
        self._ws = {}

    @classmethod
    def tfim_chain(cls, N: int, periodic: bool, J: float, Gamma: float, layers: int, d_model: int, heads: int,
                   K: int, weights: np.ndarray) -> "VQNQS":
        """The transverse-field Ising chain of N sites: vqnqs_create_tfim(N, periodic, J, Gamma, ...)."""
        self = cls.__new__(cls)
        self.L, self.N = None, N
        self.periodic, self.J, self.Gamma = bool(periodic), float(J), float(Gamma)
        self.layers, self.d, self.heads, self.K = layers, d_model, heads, K
        self.vq_heads, self.half_block, self.token_group = 1, False, 1
        w = np.ascontiguousarray(weights, dtype=np.float32)
        n = lib().vqnqs_num_params(N, layers, d_model, K)
        if w.size != n:
            raise ValueError(f"weight blob has {w.size} floats, layout needs {n}")
        h = ctypes.c_void_p()
        rc = lib().vqnqs_create_tfim(N, int(periodic), float(J), float(Gamma), layers, d_model, heads, K,
                                     w.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h))
        if rc != 0:
            raise VQNQSError(f"vqnqs_create_tfim failed: {_lib.STATUS_NAMES.get(rc, rc)}")
        self._h = h
        self._ws = {}
        return self

    def close(self):
        if getattr(self, "_h", None):
            lib().vqnqs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int, what: str):
        if rc != 0:
            msg = lib().vqnqs_last_error(self._h).decode()
            raise VQNQSError(f"{what}: {_lib.STATUS_NAMES.get(rc, rc)}: {msg}")

    def workspace_bytes(self, flags: int = 0, chunk_samples: int = 0) -> int:
        return int(lib().vqnqs_workspace_bytes(self._h, int(chunk_samples), int(flags)))

    def workspace(self, flags: int = 0, chunk_samples: int = 0) -> torch.Tensor:
        key = (flags, chunk_samples)
        if key not in self._ws:
            self._ws[key] = torch.empty(self.workspace_bytes(flags, chunk_samples), dtype=torch.uint8,
                                        device="cuda")
        return self._ws[key]

    def set_weights(self, weights, stream=None):
        if isinstance(weights, torch.Tensor):
            _check_dev(weights, torch.float32, "weights")
            self._check(lib().vqnqs_set_weights(self._h, ctypes.c_void_p(weights.data_ptr()), 1,
                                                ctypes.c_void_p(_stream_ptr(stream))), "vqnqs_set_weights")
        else:
            w = np.ascontiguousarray(weights, dtype=np.float32)
            self._check(lib().vqnqs_set_weights(self._h, w.ctypes.data_as(ctypes.c_void_p), 0,
                                                ctypes.c_void_p(_stream_ptr(stream))), "vqnqs_set_weights")

    def log_psi(self, spins: torch.Tensor, flags: int = 0, out: torch.Tensor | None = None,
                workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        _check_dev(spins, torch.uint8, "spins")
        B = spins.shape[0]
        out = torch.empty(B, dtype=torch.float32, device=spins.device) if out is None else out
        ws = self.workspace(flags) if workspace is None else workspace
        self._check(lib().vqnqs_log_psi(self._h, B, ctypes.c_void_p(spins.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), int(flags),
                                        ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                        ctypes.c_void_p(_stream_ptr(stream))), "vqnqs_log_psi")
        return out

    def sample(self, uniforms: torch.Tensor, flags: int = 0, chunk_samples: int = 0, stream=None):
        """Configurations drawn from |psi|^2 with the given uniforms [B, N] (see vqnqs_sample);
        returns (spins uint8 [B, N], log psi float [B])."""
        _check_dev(uniforms, torch.float32, "uniforms")
        if uniforms.dim() != 2 or uniforms.shape[1] != self.N:
            raise ValueError(f"uniforms must be [B, {self.N}]")
        B = uniforms.shape[0]
        spins = torch.empty(B, self.N, dtype=torch.uint8, device=uniforms.device)
        lp = torch.empty(B, dtype=torch.float32, device=uniforms.device)
        n = int(lib().vqnqs_sample_workspace_bytes(self._h, int(chunk_samples or min(B, 1024)), int(flags)))
        ws = torch.empty(n, dtype=torch.uint8, device=uniforms.device)
        self._check(lib().vqnqs_sample(self._h, B, ctypes.c_void_p(uniforms.data_ptr()),
                                       ctypes.c_void_p(spins.data_ptr()), ctypes.c_void_p(lp.data_ptr()), int(flags),
                                       ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                       ctypes.c_void_p(_stream_ptr(stream))), "vqnqs_sample")
        return spins, lp

    def vmc_step(self, uniforms: torch.Tensor, lr: float, flags: int = 0, stream=None) -> dict:
        """One VMC step (see vqnqs_vmc_step); returns the drawn spins, E_loc, the applied
        gradient and the FP64 [mean, var] of E_loc (device tensors)."""
        _check_dev(uniforms, torch.float32, "uniforms")
        B = uniforms.shape[0]
        dev = uniforms.device
        out = {"spins": torch.empty(B, self.N, dtype=torch.uint8, device=dev),
               "e_loc": torch.empty(B, dtype=torch.float32, device=dev),
               "grad": torch.empty(self.num_params, dtype=torch.float32, device=dev),
               "mean_var": torch.empty(2, dtype=torch.float64, device=dev)}
        ws = torch.empty(int(lib().vqnqs_vmc_workspace_bytes(self._h, B, int(flags))), dtype=torch.uint8, device=dev)
        self._check(lib().vqnqs_vmc_step(self._h, B, ctypes.c_void_p(uniforms.data_ptr()), float(lr),
                                         ctypes.c_void_p(out["spins"].data_ptr()), ctypes.c_void_p(out["e_loc"].data_ptr()),
                                         ctypes.c_void_p(out["grad"].data_ptr()),
                                         ctypes.c_void_p(out["mean_var"].data_ptr()), int(flags),
                                         ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                         ctypes.c_void_p(_stream_ptr(stream))), "vqnqs_vmc_step")
        return out

    def weights(self, stream=None) -> torch.Tensor:
        """The current weight blob (device copy)."""
        w = torch.empty(self.num_params, dtype=torch.float32, device="cuda")
        self._check(lib().vqnqs_get_weights(self._h, ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
                    "vqnqs_get_weights")
        return w

    def codes(self, spins: torch.Tensor, flags: int = 0, workspace: torch.Tensor | None = None, stream=None):
        """(codes [B, layers, N] int32, log psi [B]) of the configurations as given (see vqnqs_codes)."""
        _check_dev(spins, torch.uint8, "spins")
        B = spins.shape[0]
        codes = torch.empty(B, self.layers, self.N // self.token_group, dtype=torch.int32, device=spins.device)
        lp = torch.empty(B, dtype=torch.float32, device=spins.device)
        ws = self.workspace(flags) if workspace is None else workspace
        self._check(lib().vqnqs_codes(self._h, B, ctypes.c_void_p(spins.data_ptr()), ctypes.c_void_p(codes.data_ptr()),
                                      ctypes.c_void_p(lp.data_ptr()), int(flags), ctypes.c_void_p(ws.data_ptr()),
                                      ws.numel(), ctypes.c_void_p(_stream_ptr(stream))), "vqnqs_codes")
        return codes, lp

    def local_energy(self, spins: torch.Tensor, flags: int = 0, want_mean_var: bool = False,
                     want_log_psi: bool = False, out: torch.Tensor | None = None,
                     workspace: torch.Tensor | None = None, stream=None):
        """Returns e_loc [B] (and the FP64 [mean, var] and log psi when asked)."""
        _check_dev(spins, torch.uint8, "spins")
        if spins.dim() != 2 or spins.shape[1] != self.N:
            raise ValueError(f"spins must be [B, {self.N}]")
        B = spins.shape[0]
        dev = spins.device
        e = torch.empty(B, dtype=torch.float32, device=dev) if out is None else out
        mv = torch.empty(2, dtype=torch.float64, device=dev) if want_mean_var else None
        lp = torch.empty(B, dtype=torch.float32, device=dev) if want_log_psi else None
        ws = self.workspace(flags) if workspace is None else workspace
        self._check(lib().vqnqs_local_energy(
            self._h, B, ctypes.c_void_p(spins.data_ptr()), ctypes.c_void_p(e.data_ptr()),
            ctypes.c_void_p(mv.data_ptr() if mv is not None else 0),
            ctypes.c_void_p(lp.data_ptr() if lp is not None else 0), int(flags),
            ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.c_void_p(_stream_ptr(stream))),
            "vqnqs_local_energy")
        res = [e]
        if want_mean_var:
            res.append(mv)
        if want_log_psi:
            res.append(lp)
        return res[0] if len(res) == 1 else tuple(res)

    def local_energy_codes(self, spins: torch.Tensor, flags: int = 0, workspace: torch.Tensor | None = None,
                           stream=None):
        """Returns (e_loc [B], codes int32 [B, 1 + max_conn, layers, N]): the codeword of every row and
        layer of the sample (index 0) and of its connected configurations in bond order
        (vqnqs_local_energy_codes); slots of configurations a sample does not have hold -1."""
        _check_dev(spins, torch.uint8, "spins")
        if spins.dim() != 2 or spins.shape[1] != self.N:
            raise ValueError(f"spins must be [B, {self.N}]")
        B = spins.shape[0]
        n_b = 2 * self.N if self.periodic else 2 * self.L * (self.L - 1)
        if self.L is None:  # the Ising chain: one flip per site
            n_b = self.N
        e = torch.empty(B, dtype=torch.float32, device=spins.device)
        codes = torch.full((B, 1 + n_b, self.layers, self.N // self.token_group), -1, dtype=torch.int32,
                           device=spins.device)
        ws = self.workspace(flags) if workspace is None else workspace
        self._check(lib().vqnqs_local_energy_codes(
            self._h, B, ctypes.c_void_p(spins.data_ptr()), ctypes.c_void_p(e.data_ptr()),
            ctypes.c_void_p(codes.data_ptr()), int(flags), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
            ctypes.c_void_p(_stream_ptr(stream))), "vqnqs_local_energy_codes")
        return e, codes

    def _ragged_flat(self, Ls, Bs, spins, e, mv, flags, ws, stream=None):
        arr = lambda v: (ctypes.c_int * len(v))(*v)
        self._check(lib().vqnqs_local_energy_ragged(
            self._h, len(Ls), arr(Ls), arr(Bs), ctypes.c_void_p(spins.data_ptr()), ctypes.c_void_p(e.data_ptr()),
            ctypes.c_void_p(mv.data_ptr() if mv is not None else 0), int(flags), ctypes.c_void_p(ws.data_ptr()),
            ws.numel(), ctypes.c_void_p(_stream_ptr(stream))), "vqnqs_local_energy_ragged")

    def local_energy_ragged(self, groups, flags: int = 0, want_mean_var: bool = False,
                            workspace: torch.Tensor | None = None, stream=None):
        """groups: list of (L_g, spins_g [B_g, L_g^2] uint8 CUDA tensor).  Returns E_loc of all
        samples concatenated in group order (and the FP64 [mean, var])."""
        Ls = [int(L) for L, _ in groups]
        Bs = [int(s.shape[0]) for _, s in groups]
        for (L, s) in groups:
            _check_dev(s, torch.uint8, "spins")
            if s.shape[1] != L * L:
                raise ValueError("spins of a group must be [B_g, L_g^2]")
        spins = torch.cat([s.reshape(-1) for _, s in groups]).contiguous()
        total = sum(Bs)
        e = torch.empty(total, dtype=torch.float32, device=spins.device)
        mv = torch.empty(2, dtype=torch.float64, device=spins.device) if want_mean_var else None
        ws = self.workspace(flags) if workspace is None else workspace
        self._ragged_flat(Ls, Bs, spins, e, mv, flags, ws, stream)
        return (e, mv) if want_mean_var else e

    def autotune(self, M: int = 16384, stream=None) -> dict:
        """Pick the fastest tensor-core GEMM tile widths for this model (see vqnqs_autotune)."""
        t = _lib.Tuning()
        ws = torch.empty(M * self.d * 40 + 4096, dtype=torch.uint8, device="cuda")
        self._check(lib().vqnqs_autotune(self._h, int(M), ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.byref(t),
                                         ctypes.c_void_p(_stream_ptr(stream))), "vqnqs_autotune")
        return {"qkv_bn": t.qkv_bn, "mlp_up_bn": t.mlp_up_bn, "mlp_down_bn": t.mlp_down_bn,
                "ms": [[t.ms[s][i] for i in range(4)] for s in range(3)]}

    def autotune_chunk(self, spins: torch.Tensor, flags: int = 0, candidates=(8, 15, 30, 60), stream=None) -> dict:
        """Times the local energies of ``spins`` at each candidate chunk size (samples per
        chunk; see vqnqs_autotune_chunk) and returns {"best": samples, "ms": {size: ms}}."""
        _check_dev(spins, torch.uint8, "spins")
        cand = [int(c) for c in candidates]
        ws = self.workspace(flags, max(cand))
        arr = (ctypes.c_int * len(cand))(*cand)
        ms = (ctypes.c_float * len(cand))()
        best = ctypes.c_int()
        self._check(lib().vqnqs_autotune_chunk(self._h, spins.shape[0], ctypes.c_void_p(spins.data_ptr()), int(flags),
                                               arr, len(cand), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                               ctypes.byref(best), ms, ctypes.c_void_p(_stream_ptr(stream))),
                    "vqnqs_autotune_chunk")
        return {"best": best.value, "ms": {c: float(ms[i]) for i, c in enumerate(cand)}}

    def autotune_incremental(self, spins: torch.Tensor, flags: int, chunk_samples: int = 0, stream=None) -> dict:
        """Picks the incremental path's work split (patch items per CTA, changed-row items per
        SM; see vqnqs_autotune_incremental) by timing the local energies of ``spins`` with
        ``flags`` (chunks of ``chunk_samples``, 0: the default), keeps it for this model and returns
        {"patch_items", "rows_slices", "patch_ms": {items: ms}, "rows_ms": {items: ms}}."""
        _check_dev(spins, torch.uint8, "spins")
        ws = self.workspace(flags, chunk_samples)
        t = _lib.IncTuning()
        self._check(lib().vqnqs_autotune_incremental(self._h, spins.shape[0], ctypes.c_void_p(spins.data_ptr()),
                                                     int(flags), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                                     ctypes.byref(t), ctypes.c_void_p(_stream_ptr(stream))),
                    "vqnqs_autotune_incremental")
        return {"patch_items": t.patch_items, "rows_slices": t.rows_slices,
                "patch_ms": {n: float(t.patch_ms[i]) for i, n in enumerate((2, 4, 8))},
                "rows_ms": {n: float(t.rows_ms[i]) for i, n in enumerate((1, 2, 4, 8, 16))}}

    def stats(self) -> dict:
        s = _lib.Stats()
        self._check(lib().vqnqs_get_stats(self._h, ctypes.byref(s)), "vqnqs_get_stats")
        return {
            "samples": s.samples, "configs": s.configs, "rows": s.rows,
            "unique_rows": [int(s.unique_rows[i]) for i in range(self.layers + 1)],
            "near_ties": s.near_ties, "flops_full": s.flops_full, "flops_done": s.flops_done,
            "device_status": s.device_status, "active_rows": s.active_rows, "attn_pairs": s.attn_pairs,
            "inc_base_rows": s.inc_base_rows, "inc_patched_rows": s.inc_patched_rows,
            "inc_certified_rows": s.inc_certified_rows, "inc_full_rows": s.inc_full_rows,
            "inc_searched_rows": s.inc_searched_rows, "inc_patch_pairs": s.inc_patch_pairs,
            "inc_full_pairs": s.inc_full_pairs, "inc_whole_pairs": s.inc_whole_pairs,
        }

    def check_timeout_path(self, limit_cycles: int = 1_000_000, stream=None):
        """Run the bounded-wait failure probe (see vqnqs_check_timeout_path)."""
        self._check(lib().vqnqs_check_timeout_path(self._h, int(limit_cycles), ctypes.c_void_p(_stream_ptr(stream))),
                    "vqnqs_check_timeout_path")

    def reset_stats(self):
        self._check(lib().vqnqs_reset_stats(self._h), "vqnqs_reset_stats")

    def profile(self, enable: bool = True):
        self._check(lib().vqnqs_profile_enable(self._h, int(enable)), "vqnqs_profile_enable")

    def profile_read(self) -> dict:
        """{stage: (calls, launches, ms)} since the last read."""
        arr = (_lib.StageTime * _lib.MAX_STAGES)()
        n = ctypes.c_int()
        self._check(lib().vqnqs_profile_read(self._h, arr, _lib.MAX_STAGES, ctypes.byref(n)), "vqnqs_profile_read")
        return {arr[i].name.decode(): (int(arr[i].calls), int(arr[i].launches), float(arr[i].ms))
                for i in range(n.value)}

    def launch_count(self) -> int:
        return int(lib().vqnqs_launch_count(self._h))

    def gemm_bf16(self, A: torch.Tensor, Bt: torch.Tensor, bias: torch.Tensor, epilogue: int = 3,
                  R: torch.Tensor | None = None, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """C = A @ Bt^T + bias with the library's tensor-core GEMM (see vqnqs_gemm_bf16)."""
        _check_dev(A, torch.bfloat16, "A")
        _check_dev(Bt, torch.bfloat16, "Bt")
        _check_dev(bias, torch.float32, "bias")
        M, K = A.shape
        N = Bt.shape[0]
        if out is None:
            out = torch.empty(M, N, dtype=torch.bfloat16 if epilogue in (0, 1) else torch.float32, device=A.device)
        if R is not None:
            _check_dev(R, torch.float32, "R")
        self._check(lib().vqnqs_gemm_bf16(self._h, M, N, K, ctypes.c_void_p(A.data_ptr()),
                                          ctypes.c_void_p(Bt.data_ptr()), ctypes.c_void_p(bias.data_ptr()),
                                          ctypes.c_void_p(R.data_ptr() if R is not None else 0),
                                          ctypes.c_void_p(out.data_ptr()), int(epilogue),
                                          ctypes.c_void_p(_stream_ptr(stream))), "vqnqs_gemm_bf16")
        return out

    def gemm_bf16_split(self, A2: torch.Tensor, Bt2: torch.Tensor, bias: torch.Tensor, epilogue: int = 3,
                        R: torch.Tensor | None = None, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """C = A @ Bt^T + bias from split operands A2 = [A_hi; A_lo] [2M, K], Bt2 = [Bt_hi; Bt_lo]
        [2N, K] (see vqnqs_gemm_bf16_split); BF16 outputs come back as [2M, N] (hi rows, then lo rows)."""
        _check_dev(A2, torch.bfloat16, "A2")
        _check_dev(Bt2, torch.bfloat16, "Bt2")
        _check_dev(bias, torch.float32, "bias")
        M, K = A2.shape[0] // 2, A2.shape[1]
        N = Bt2.shape[0] // 2
        if out is None:
            out = (torch.empty(2 * M, N, dtype=torch.bfloat16, device=A2.device) if epilogue in (0, 1) else
                   torch.empty(M, N, dtype=torch.float32, device=A2.device))
        if R is not None:
            _check_dev(R, torch.float32, "R")
        self._check(lib().vqnqs_gemm_bf16_split(self._h, M, N, K, ctypes.c_void_p(A2.data_ptr()),
                                                ctypes.c_void_p(Bt2.data_ptr()), ctypes.c_void_p(bias.data_ptr()),
                                                ctypes.c_void_p(R.data_ptr() if R is not None else 0),
                                                ctypes.c_void_p(out.data_ptr()), int(epilogue),
                                                ctypes.c_void_p(_stream_ptr(stream))), "vqnqs_gemm_bf16_split")
        return out

    def compress_rows(self, uid: torch.Tensor, code: torch.Tensor, stream=None):
        """Dense new ids of the distinct (uid, code) pairs (see vqnqs_compress_rows).

        Returns (new_id [R], rep_uid [R], rep_code [R], count [1]) device tensors."""
        _check_dev(uid, torch.int32, "uid")
        _check_dev(code, torch.int32, "code")
        R = uid.numel()
        dev = uid.device
        new_id = torch.empty(R, dtype=torch.int32, device=dev)
        rep_uid = torch.empty(R, dtype=torch.int32, device=dev)
        rep_code = torch.empty(R, dtype=torch.int32, device=dev)
        count = torch.empty(1, dtype=torch.int32, device=dev)
        ws = torch.empty(int(lib().vqnqs_compress_workspace_bytes(R)), dtype=torch.uint8, device=dev)
        ptr = lambda t: ctypes.c_void_p(t.data_ptr())
        self._check(lib().vqnqs_compress_rows(self._h, R, ptr(uid), ptr(code), ptr(new_id), ptr(rep_uid),
                                              ptr(rep_code), ptr(count), ptr(ws), ws.numel(),
                                              ctypes.c_void_p(_stream_ptr(stream))), "vqnqs_compress_rows")
        return new_id, rep_uid, rep_code, count

    @property
    def num_params(self) -> int:
        return int(lib().vqnqs_num_params_arch(self.N, self.layers, self.d, self.K, int(self.half_block),
                                               self.token_group))

    def grad_log_psi(self, spins: torch.Tensor, seeds: torch.Tensor | None = None,
                     e_loc: torch.Tensor | None = None, want_O: bool = False, want_grad: bool = True,
                     chunk_samples: int = 0, flags: int = 0, stream=None):
        """(O [B, P] or None, grad [P] or None); see vqnqs_grad_log_psi (flags: BF16 puts the summed
        gradient's contractions on the tensor cores with split operands)."""
        _check_dev(spins, torch.uint8, "spins")
        B = spins.shape[0]
        P = self.num_params
        dev = spins.device
        O = torch.empty(B, P, dtype=torch.float32, device=dev) if want_O else None
        grad = torch.empty(P, dtype=torch.float32, device=dev) if want_grad else None
        for t, name in ((seeds, "seeds"), (e_loc, "e_loc")):
            if t is not None:
                _check_dev(t, torch.float32, name)
        ws = torch.empty(int(lib().vqnqs_grad_workspace_bytes(self._h, B, int(chunk_samples))), dtype=torch.uint8,
                         device=dev)
        ptr = lambda t: ctypes.c_void_p(t.data_ptr() if t is not None else 0)
        self._check(lib().vqnqs_grad_log_psi(self._h, B, ptr(spins), ptr(seeds), ptr(e_loc), ptr(O), ptr(grad),
                                             int(flags),
                                             ptr(ws), ws.numel(), ctypes.c_void_p(_stream_ptr(stream))),
                    "vqnqs_grad_log_psi")
        return O, grad

    def energy_grad_partials(self, spins: torch.Tensor, e_loc: torch.Tensor, chunk_samples: int = 0,
                             flags: int = 0, stream=None) -> torch.Tensor:
        """This rank's FP64 partial sums [2P + 3] of the sharded energy gradient
        (sum E O, sum O, sum E, sum E^2, n; see vqnqs_energy_grad_partials)."""
        _check_dev(spins, torch.uint8, "spins")
        _check_dev(e_loc, torch.float32, "e_loc")
        B = spins.shape[0]
        P = self.num_params
        part = torch.empty(2 * P + 3, dtype=torch.float64, device=spins.device)
        ws = torch.empty(int(lib().vqnqs_energy_grad_partials_workspace_bytes(self._h, B, int(chunk_samples))),
                         dtype=torch.uint8, device=spins.device)
        self._check(lib().vqnqs_energy_grad_partials(self._h, B, ctypes.c_void_p(spins.data_ptr()),
                                                     ctypes.c_void_p(e_loc.data_ptr()), ctypes.c_void_p(part.data_ptr()),
                                                     int(flags), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                                     ctypes.c_void_p(_stream_ptr(stream))),
                    "vqnqs_energy_grad_partials")
        return part

    def energy_grad_combine(self, partials: torch.Tensor, stream=None):
        """(grad [P] float32, [mean, var] float64) from the all-reduced partials
        (see vqnqs_energy_grad_combine)."""
        _check_dev(partials, torch.float64, "partials")
        grad = torch.empty(self.num_params, dtype=torch.float32, device=partials.device)
        mv = torch.empty(2, dtype=torch.float64, device=partials.device)
        self._check(lib().vqnqs_energy_grad_combine(self._h, ctypes.c_void_p(partials.data_ptr()),
                                                    ctypes.c_void_p(grad.data_ptr()), ctypes.c_void_p(mv.data_ptr()),
                                                    ctypes.c_void_p(_stream_ptr(stream))),
                    "vqnqs_energy_grad_combine")
        return grad, mv

    def vq_assign(self, layer: int, O: torch.Tensor, tensor_cores: bool = False, stream=None) -> torch.Tensor:
        """Nearest codeword of each row of O under layer `layer`'s codebook (see vqnqs_vq_assign)."""
        _check_dev(O, torch.float32, "O")
        R = O.shape[0]
        code = torch.empty(R, dtype=torch.int32, device=O.device)
        self._check(lib().vqnqs_vq_assign(self._h, int(layer), R, ctypes.c_void_p(O.data_ptr()),
                                          ctypes.c_void_p(code.data_ptr()), int(tensor_cores),
                                          ctypes.c_void_p(_stream_ptr(stream))), "vqnqs_vq_assign")
        return code


class LogPsi(torch.autograd.Function):
    """log psi(spins) as a differentiable function of the flat weight blob.

    forward: uploads the weights into the model (vqnqs_set_weights) and calls
    vqnqs_log_psi; backward: vqnqs_grad_log_psi seeded with the incoming
    gradient, i.e. the hand-written straight-through backward with activation
    recomputation."""

    @staticmethod
    def forward(ctx, weights: torch.Tensor, spins: torch.Tensor, model: VQNQS, flags: int = 0):
        model.set_weights(weights.detach().contiguous())
        lp = model.log_psi(spins, flags)
        ctx.save_for_backward(spins)
        ctx.model = model
        return lp

    @staticmethod
    def backward(ctx, g):
        (spins,) = ctx.saved_tensors
        _, grad = ctx.model.grad_log_psi(spins, seeds=g.detach().float().contiguous())
        return grad, None, None, None


class LocalEnergyGraph:
    """A local-energy evaluation of fixed shape captured into one CUDA graph.

    ``shapes`` is a list of (L, B) lattice groups: one group with the model's
    own L uses vqnqs_local_energy, several use vqnqs_local_energy_ragged.  Call
    with one spins tensor per group; the spins are copied into the graph's
    input buffer, the graph is replayed, and the E_loc buffer is returned (valid
    until the next call).  The first, uncaptured evaluation performs every
    one-time set-up (kernel attributes, module loading) before capture.
    ``chunk_samples`` sizes the workspace (vqnqs_workspace_bytes; 0: the default)."""

    def __init__(self, model: VQNQS, shapes, flags: int = 0, chunk_samples: int = 0):
        self.model, self.flags = model, int(flags)
        self.Ls = [int(L) for L, _ in shapes]
        self.Bs = [int(B) for _, B in shapes]
        self.uniform = len(shapes) == 1 and self.Ls[0] == model.L
        total_sites = sum(L * L * B for L, B in zip(self.Ls, self.Bs))
        self.spins = torch.zeros(total_sites, dtype=torch.uint8, device="cuda")
        self.out = torch.empty(sum(self.Bs), dtype=torch.float32, device="cuda")
        self.ws = torch.empty(model.workspace_bytes(self.flags, chunk_samples), dtype=torch.uint8, device="cuda")
        self._run()
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            with torch.cuda.graph(self.graph, stream=side):
                self._run()
        torch.cuda.current_stream().wait_stream(side)

    def _run(self):
        if self.uniform:
            self.model.local_energy(self.spins.view(self.Bs[0], -1), self.flags, out=self.out, workspace=self.ws)
        else:
            self.model._ragged_flat(self.Ls, self.Bs, self.spins, self.out, None, self.flags, self.ws)

    def __call__(self, *spins):
        off = 0
        for s, L, B in zip(spins, self.Ls, self.Bs):
            n = L * L * B
            self.spins[off:off + n].copy_(s.reshape(-1), non_blocking=True)
            off += n
        self.graph.replay()
        return self.out
