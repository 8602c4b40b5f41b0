"""Python face of the C ABI: handle classes and tensor-level calls.

Each function marshals arguments (torch tensors -> device pointers, the
current CUDA stream) and calls the C entry point of the same name; all
computation happens in the library's kernels.  Layouts are those of
include/satsampler.h: V, m, v, gV are [n_pi, B] float32; act/adj are
tile-major [ceil(B/128), n_cone, 128]; bit arrays are [rows, ceil(B/32)] int32
words.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _native as N
from ._native import check, lib


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def round32(x: int) -> int:
    return (x + 31) // 32 * 32


class _Handle:
    _free = None

    def __init__(self, h):
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            getattr(lib(), self._free)(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Cnf(_Handle):
    _free = "sat_cnf_free"

    @classmethod
    def from_dimacs(cls, text: str | bytes) -> "Cnf":
        b = text.encode() if isinstance(text, str) else text
        h = C.c_void_p()
        check(lib().sat_cnf_from_dimacs(b, len(b), C.byref(h)))
        return cls(h)

    @classmethod
    def from_file(cls, path: str) -> "Cnf":
        h = C.c_void_p()
        check(lib().sat_cnf_from_file(str(path).encode(), C.byref(h)))
        return cls(h)

    def info(self):
        nv, nc, nl = C.c_uint32(), C.c_uint64(), C.c_uint64()
        check(lib().sat_cnf_info(self._h, C.byref(nv), C.byref(nc), C.byref(nl)))
        return nv.value, nc.value, nl.value


def _struct_dict(s):
    return {name: getattr(s, name) for name, _ in s._fields_}


class Circuit(_Handle):
    _free = "sat_circuit_free"

    @classmethod
    def build(cls, cnf: Cnf, max_support: int = 8, max_window: int = 16, direct: bool = False,
              reorder: bool = False):
        """Algorithm 1 (default), or with direct=True one OR output per clause and no
        factorization (the direct relaxation the paper compares against).  reorder=True
        sorts the clauses by (largest variable, position) first, for files whose gate
        clauses are not adjacent."""
        h = C.c_void_p()
        st = N.BuildStats()
        opts = N.BuildOpts(max_support, max_window, 1 if direct else 0, 1 if reorder else 0)
        check(lib().sat_circuit_build(cnf.handle, C.byref(opts), C.byref(h), C.byref(st)))
        c = cls(h)
        c.stats = _struct_dict(st)
        return c

    def dump(self) -> str:
        n = C.c_size_t()
        check(lib().sat_circuit_dump(self._h, None, 0, C.byref(n)))
        buf = C.create_string_buffer(n.value + 1)
        check(lib().sat_circuit_dump(self._h, buf, n.value + 1, C.byref(n)))
        return buf.value.decode()

    def round_program(self, compile: bool = False) -> str:
        """The generated CUDA program of the circuit's instance-compiled round kernel, or with
        compile the NVRTC log of compiling it for sm_103a (host only; raises for a circuit
        beyond the kernel's limits or a failed compilation)."""
        n = C.c_size_t()
        check(lib().sat_circuit_round_program(self._h, int(compile), None, 0, C.byref(n)))
        buf = C.create_string_buffer(n.value + 1)
        check(lib().sat_circuit_round_program(self._h, int(compile), buf, n.value + 1, C.byref(n)))
        return buf.value.decode()


class Plan(_Handle):
    _free = "sat_plan_free"

    @classmethod
    def create(cls, circuit: Circuit, cnf: Cnf) -> "Plan":
        h = C.c_void_p()
        check(lib().sat_plan_create(circuit.handle, cnf.handle, C.byref(h)))
        p = cls(h)
        info = N.PlanInfo()
        check(lib().sat_plan_get_info(h, C.byref(info)))
        p.info = _struct_dict(info)
        return p

    def __getattr__(self, k):
        info = self.__dict__.get("info")
        if info is not None and k in info:
            return info[k]
        raise AttributeError(k)

    def status(self, clear: bool = True, stream=None) -> int:
        """Kernel status word (0 = healthy; bit 2 = an async-copy wait expired)."""
        v = C.c_uint32()
        check(lib().sat_plan_status(self._h, C.byref(v), int(clear), _stream(stream)))
        return v.value

    STEP_KERNELS = {"auto": 0, "tiled": 1, "resident": 2}
    ACT_CODES = {"f32": 0, "bf16": 1, "f16": 2}

    def set_step_kernel(self, kind: str = "auto") -> None:
        """Kernel of the fused steps: "tiled", "resident" (shared-memory resident, for
        circuits that fit) or "auto" (resident when it fits)."""
        check(lib().sat_plan_set_step_kernel(self._h, self.STEP_KERNELS[kind]))

    def step_kernel(self, act_dtype: str = "f32") -> str:
        """The kernel ("tiled" or "resident") that a step call with act_dtype would use."""
        k = C.c_int32()
        check(lib().sat_plan_step_kernel(self._h, self.ACT_CODES[act_dtype], C.byref(k)))
        return {1: "tiled", 2: "resident"}[k.value]

    def round_info(self, compile: bool = False) -> dict:
        """The plan's instance-compiled round kernel: available, compiled, registers,
        spill_bytes, min_blocks, compile_ms (compile: compile and load it now)."""
        r = N.RoundInfo()
        check(lib().sat_plan_round_info(self._h, int(compile), C.byref(r)))
        return {k: getattr(r, k) for k, _ in r._fields_}

    def scratch_elems(self, B: int) -> int:
        n = C.c_uint64()
        check(lib().sat_plan_scratch_elems(self._h, B, C.byref(n)))
        return n.value

    def layout_rows(self, segment: int = 0):
        """Rows per 128-sample tile of the act scratch (recomputation segment `segment`,
        0 = every level stored) and of the adj scratch (the adjoint ring)."""
        a, g = C.c_uint64(), C.c_uint64()
        check(lib().sat_plan_layout_elems(self._h, segment, N.TILE, C.byref(a), C.byref(g)))
        return a.value // N.TILE, g.value // N.TILE

    def pi_vars(self) -> np.ndarray:
        out = np.zeros(self.info["n_pi"], np.uint32)
        check(lib().sat_plan_pi_vars(self._h, out.ctypes.data_as(C.c_void_p)))
        return out

    def var_nodes(self):
        n = self.info["n_vars"] + 1
        cone = np.zeros(n, np.int64)
        full = np.zeros(n, np.int64)
        neg = np.zeros(n, np.uint8)
        check(lib().sat_plan_var_nodes(self._h, cone.ctypes.data_as(C.c_void_p), full.ctypes.data_as(C.c_void_p),
                                       neg.ctypes.data_as(C.c_void_p)))
        return cone, full, neg


class Dedup(_Handle):
    _free = "sat_dedup_free"

    @classmethod
    def create(cls, plan: Plan, max_keys: int, max_batch: int) -> "Dedup":
        h = C.c_void_p()
        check(lib().sat_dedup_create(plan.handle, max_keys, max_batch, C.byref(h)))
        d = cls(h)
        d.key_words = plan.info["key_words"]
        d.max_batch = max_batch
        return d

    def insert(self, keys, valid, B: int, hashes=None, is_new=None, stream=None, sync=True):
        """Insert a batch; sync=False skips the host synchronisations (sat_dedup_insert_async:
        failures are reported later by check())."""
        if not sync:
            assert hashes is None and is_new is None
            check(lib().sat_dedup_insert_async(self._h, _ptr(keys), _ptr(valid), B, _stream(stream)))
            return
        check(lib().sat_dedup_insert(self._h, _ptr(keys), _ptr(valid), B, _ptr(hashes), _ptr(is_new),
                                     _stream(stream)))

    def check(self, stream=None) -> None:
        """Raise SatError(SAT_ERR_TABLE_FULL) if any insert so far did not fit."""
        check(lib().sat_dedup_check(self._h, _stream(stream)))

    def count(self, stream=None) -> int:
        n = C.c_uint64()
        check(lib().sat_dedup_count(self._h, C.byref(n), _stream(stream)))
        return n.value

    def keys(self, stream=None) -> np.ndarray:
        n = self.count(stream)
        out = np.zeros((n, self.key_words), np.uint32)
        check(lib().sat_dedup_copy_keys(self._h, 0, n, out.ctypes.data_as(C.c_void_p), _stream(stream)))
        return out

    def clear(self, stream=None):
        check(lib().sat_dedup_clear(self._h, _stream(stream)))


class Solutions(_Handle):
    _free = "sat_solutions_free"

    def __len__(self):
        return lib().sat_solutions_count(self._h)

    @property
    def n_vars(self):
        return lib().sat_solutions_nvars(self._h)

    def words(self, first: int = 0, count: int | None = None) -> np.ndarray:
        n = len(self) - first if count is None else count
        nw = (self.n_vars + 63) // 64
        out = np.zeros((n, nw), np.uint64)
        check(lib().sat_solutions_copy(self._h, first, n, out.ctypes.data_as(C.c_void_p)))
        return out

    def assignments(self) -> np.ndarray:
        """[count, n_vars] 0/1 array (variable v in column v-1)."""
        w = self.words()
        bits = np.unpackbits(w.view(np.uint8), axis=1, bitorder="little")
        return bits[:, : self.n_vars]


class Mlp(_Handle):
    """The learned proposal network (see sat_mlp_* in include/satsampler.h)."""
    _free = "sat_mlp_free"

    @classmethod
    def create(cls, n_in: int, n_hidden: int, n_out: int, max_rows: int, seed: int = 0) -> "Mlp":
        h = C.c_void_p()
        check(lib().sat_mlp_create(n_in, n_hidden, n_out, max_rows, seed, C.byref(h)))
        m = cls(h)
        m.n_in, m.n_hidden, m.n_out, m.max_rows = n_in, n_hidden, n_out, max_rows
        n = C.c_uint64()
        check(lib().sat_mlp_num_params(h, C.byref(n)))
        m.n_params = n.value
        return m

    def params(self) -> np.ndarray:
        out = np.zeros(self.n_params, np.float32)
        check(lib().sat_mlp_get_params(self._h, out.ctypes.data_as(C.c_void_p)))
        return out

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        assert th.size == self.n_params
        check(lib().sat_mlp_set_params(self._h, th.ctypes.data_as(C.c_void_p)))

    def draw_noise(self, rows: int, seed: int, round_: int = 0, device="cuda", stream=None):
        import torch
        z = torch.empty((rows, self.n_in), dtype=torch.bfloat16, device=device)
        check(lib().sat_mlp_draw_noise(self._h, seed, round_, _ptr(z), rows, _stream(stream)))
        return z

    def forward(self, z, tau: float = 1.0, V=None, stream=None):
        """tau * logits as [n_out, rows] float32 (the sampler's V layout)."""
        import torch
        rows = z.shape[0]
        if V is None:
            V = torch.empty((self.n_out, rows), dtype=torch.float32, device=z.device)
        check(lib().sat_mlp_forward(self._h, _ptr(z), rows, tau, _ptr(V), V.stride(0), _stream(stream)))
        return V

    def propose(self, V, seed: int, round_: int, tau: float = 1.0, stream=None):
        check(lib().sat_mlp_propose(self._h, seed, round_, tau, _ptr(V), V.stride(0), V.shape[1], _stream(stream)))

    def imle_select(self, zc, keys, S: int, K: int, stream=None):
        import torch
        dist = torch.empty(S * K, dtype=torch.float32, device=zc.device)
        choice = torch.empty(S, dtype=torch.int32, device=zc.device)
        check(lib().sat_mlp_imle_select(self._h, _ptr(zc), _ptr(keys), keys.shape[1], S, K, _ptr(dist), _ptr(choice),
                                        _stream(stream)))
        return dist, choice

    def loss_grad(self, z, keys, stream=None):
        S = z.shape[0]
        loss = C.c_float()
        g = np.zeros(self.n_params, np.float32)
        check(lib().sat_mlp_loss_grad(self._h, _ptr(z), _ptr(keys), keys.shape[1], S, C.byref(loss),
                                      g.ctypes.data_as(C.c_void_p), _stream(stream)))
        return loss.value, g

    def train(self, plan: "Plan", solutions, steps: int, S: int = 4096, K: int = 16, lr: float = 1e-3,
              seed: int = 0, stream=None) -> float:
        """IMLE training on distinct solutions (sat_mlp_train): `solutions` is a uint64 array
        [n, ceil(n_vars/64)] of full assignments (Solutions.words() format) of plan's circuit.
        Returns the last step's mean loss."""
        w = np.ascontiguousarray(solutions, dtype=np.uint64)
        loss = C.c_float()
        check(lib().sat_mlp_train(self._h, plan.handle, w.ctypes.data, w.shape[0], steps, S, K, lr, seed,
                                  C.byref(loss), _stream(stream)))
        return float(loss.value)

    def apply_grad(self, grad, lr: float, stream=None) -> None:
        """One Adam step with a given gradient (device float32 [n_params]; sat_mlp_apply_grad)."""
        check(lib().sat_mlp_apply_grad(self._h, _ptr(grad), lr, _stream(stream)))

    def train_step(self, keys, S: int, K: int, lr: float, seed: int, round_: int, stream=None) -> float:
        loss = C.c_float()
        check(lib().sat_mlp_train_step(self._h, _ptr(keys), keys.shape[1], S, K, lr, seed, round_, C.byref(loss),
                                       _stream(stream)))
        return loss.value

    def status(self) -> int:
        v = C.c_uint32()
        check(lib().sat_mlp_status(self._h, C.byref(v)))
        return v.value


# --------------------------------------------------------- kernel calls ---
def opt_params(optimizer="adam", lr=0.1, beta1=0.9, beta2=0.999, eps=1e-8) -> N.OptParams:
    return N.OptParams(N.OPTIMIZERS[optimizer], lr, beta1, beta2, eps)


def _act_torch_dtype(act_dtype: str):
    import torch
    return {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[act_dtype]


def _tiles(B: int) -> int:
    return (B + N.TILE - 1) // N.TILE


def new_act(plan: Plan, B: int, act_dtype: str = "f32", device="cuda", segment: int = 0):
    """act scratch [tiles][rows][128]: rows = n_cone (segment 0, every level stored; the
    layout sat_forward writes) or the rows of recomputation segment `segment`."""
    import torch
    rows = plan.info["n_cone"] if segment == 0 else plan.layout_rows(segment)[0]
    return torch.empty((_tiles(B), rows, N.TILE), dtype=_act_torch_dtype(act_dtype), device=device)


def new_adj(plan: Plan, B: int, device="cuda"):
    """adj scratch [tiles][rows][128] (the input level plus a ring of max_span + 1 gate levels)."""
    import torch
    return torch.empty((_tiles(B), plan.layout_rows(0)[1], N.TILE), dtype=torch.float32, device=device)


def untile(x, B: int):
    """[n_cone, B] view of a tile-major act array of the full layout."""
    return x.permute(1, 0, 2).reshape(x.shape[1], -1)[:, :B]


def sat_init_normal(plan: Plan, V, seed: int, round_: int = 0, scale: float = 1.0, stream=None):
    check(lib().sat_init_normal(plan.handle, seed, round_, scale, _ptr(V), V.stride(0), V.shape[1], _stream(stream)))


def sat_forward(plan: Plan, V, act, loss=None, act_dtype="f32", stream=None):
    check(lib().sat_forward(plan.handle, N.ACT_DTYPES[act_dtype], _ptr(V), V.stride(0), _ptr(act), _ptr(loss),
                            V.shape[1], _stream(stream)))


def sat_backward(plan: Plan, V, act, adj, gV, grad_loss=None, act_dtype="f32", stream=None):
    check(lib().sat_backward(plan.handle, N.ACT_DTYPES[act_dtype], _ptr(V), V.stride(0), _ptr(act), _ptr(adj),
                             _ptr(grad_loss), _ptr(gV), V.shape[1], _stream(stream)))


def sat_opt_update(plan: Plan, opt: N.OptParams, V, m, v, gV, t: int, stream=None):
    check(lib().sat_opt_update(plan.handle, C.byref(opt), _ptr(V), _ptr(m), _ptr(v), _ptr(gV), V.stride(0), t,
                               V.shape[1], _stream(stream)))


def sat_steps(plan: Plan, opt: N.OptParams, V, m, v, act, adj, t0: int, n_steps: int, loss=None,
              act_dtype="f32", stream=None, age=None, segment: int = 0):
    """Fused steps; with `age` (int32 [B]) the Adam step of sample b is age[b] + t0 + s (sat_steps_aged);
    with segment > 0, level-segment recomputation (sat_steps_recompute; act from new_act(..., segment=))."""
    if segment:
        check(lib().sat_steps_recompute(plan.handle, N.ACT_DTYPES[act_dtype], C.byref(opt), _ptr(V), _ptr(m),
                                        _ptr(v), V.stride(0), _ptr(act), _ptr(adj), _ptr(loss), _ptr(age), t0,
                                        n_steps, V.shape[1], segment, _stream(stream)))
    elif age is None:
        check(lib().sat_steps(plan.handle, N.ACT_DTYPES[act_dtype], C.byref(opt), _ptr(V), _ptr(m), _ptr(v),
                              V.stride(0), _ptr(act), _ptr(adj), _ptr(loss), t0, n_steps, V.shape[1],
                              _stream(stream)))
    else:
        check(lib().sat_steps_aged(plan.handle, N.ACT_DTYPES[act_dtype], C.byref(opt), _ptr(V), _ptr(m), _ptr(v),
                                   V.stride(0), _ptr(act), _ptr(adj), _ptr(loss), _ptr(age), t0, n_steps,
                                   V.shape[1], _stream(stream)))


def sat_retire(valid, age, restart, k: int, max_age: int, B: int, stream=None):
    check(lib().sat_retire(_ptr(valid), _ptr(age), _ptr(restart), k, max_age, B, _stream(stream)))


def sat_restart(plan: Plan, restart, seed: int, round_: int, V, m, v, scale: float = 1.0, src=None, stream=None):
    check(lib().sat_restart(plan.handle, _ptr(restart), seed, round_, scale, _ptr(src),
                            0 if src is None else src.stride(0), _ptr(V), _ptr(m), _ptr(v), V.stride(0), V.shape[1],
                            _stream(stream)))


def sat_steps_noalloc(plan: Plan, opt: N.OptParams, V, m, v, t0: int, n_steps: int, loss=None, act_dtype="f32",
                      stream=None):
    """sat_steps with the library's fixed scratch array (no act/adj buffers, no allocation)."""
    check(lib().sat_steps_noalloc(plan.handle, N.ACT_DTYPES[act_dtype], C.byref(opt), _ptr(V), _ptr(m), _ptr(v),
                                  V.stride(0), _ptr(loss), t0, n_steps, V.shape[1], _stream(stream)))


def sat_threshold(plan: Plan, V, node_bits, keys, stream=None):
    check(lib().sat_threshold(plan.handle, _ptr(V), V.stride(0), _ptr(node_bits), node_bits.stride(0), _ptr(keys),
                              V.shape[1], _stream(stream)))


def sat_hard_eval(plan: Plan, node_bits, B: int, stream=None):
    check(lib().sat_hard_eval(plan.handle, _ptr(node_bits), node_bits.stride(0), B, _stream(stream)))


def sat_cnf_check(plan: Plan, node_bits, valid, B: int, stream=None):
    check(lib().sat_cnf_check(plan.handle, _ptr(node_bits), node_bits.stride(0), _ptr(valid), B, _stream(stream)))


def sat_round_gd(plan: Plan, keys, valid, B: int, lr: float, steps: int, seed: int = 0, round_: int = 0,
                 scale: float = 1.0, V=None, stream=None):
    """One plain-GD sampling round in the plan's instance-compiled kernel: init, steps,
    threshold, Boolean pass and clause check (keys [B][key_words] int32, valid
    [ceil(B/32)] int32; V, if given, [n_pi][ldv] receives the final logits)."""
    check(lib().sat_round_gd(plan.handle, lr, steps, seed, round_, scale, _ptr(V), V.stride(0) if V is not None else 0,
                             _ptr(keys), _ptr(valid), B, _stream(stream)))


def sat_gemm_bf16(A, B, bias=None, epilogue=0, pre=None, alpha=1.0, out_f32=None, out_bf16=None, out_t_bf16=None,
                  out_t_f32=None, status=None, stream=None):
    """D = A B^T on the tensor cores with the fused epilogue (see satsampler.h)."""
    M, K = A.shape
    N = B.shape[0]
    ldo = (out_f32 if out_f32 is not None else out_bf16).stride(0) if (out_f32 is not None or out_bf16 is not None) else 0
    ldt = (out_t_bf16 if out_t_bf16 is not None else out_t_f32).stride(0) \
        if (out_t_bf16 is not None or out_t_f32 is not None) else 0
    check(lib().sat_gemm_bf16(M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(bias), epilogue, _ptr(pre),
                              0 if pre is None else pre.stride(0), alpha, _ptr(out_f32), _ptr(out_bf16), ldo,
                              _ptr(out_t_bf16), _ptr(out_t_f32), ldt, _ptr(status), _stream(stream)))


@dataclass
class Workspace:
    """Device buffers of one sampling round (torch-allocated)."""
    B: int
    V: object
    m: object
    v: object
    act: object
    adj: object
    bits: object
    keys: object
    valid: object
    loss: object
    act_dtype: str = "f32"
    age: object = None      # early exit (run_epochs): int32 [B] steps since each sample's start
    restart: object = None  # early exit: restart bits [ceil(B/32)]
    src: object = None      # early exit with a proposal: new starts [n_pi][B]
    segment: int = 0        # level-segment recomputation of the fused steps (act laid out for it)


def new_workspace(plan: Plan, B: int, act_dtype: str = "f32", device="cuda", segment: int = 0) -> Workspace:
    import torch
    npi = plan.info["n_pi"]
    W = (B + 31) // 32
    z = lambda *s: torch.zeros(s, dtype=torch.float32, device=device)
    return Workspace(
        B, z(npi, B), z(npi, B), z(npi, B), new_act(plan, B, act_dtype, device, segment), new_adj(plan, B, device),
        torch.zeros((plan.info["n_nodes"], W), dtype=torch.int32, device=device),
        torch.zeros((B, max(1, plan.info["key_words"])), dtype=torch.int32, device=device),
        torch.zeros(W, dtype=torch.int32, device=device), z(B), act_dtype, segment=segment)


def run_round(plan: Plan, ws: Workspace, opt: N.OptParams, steps: int, seed: int, round_: int,
              init_scale: float = 1.0, dedup: Dedup | None = None, init_logits=None, proposal: "Mlp | None" = None,
              tau: float = 1.0, stream=None):
    """One round on device-resident buffers: init (Philox, caller logits or the
    proposal network), steps, threshold, Boolean pass, CNF check, dedup."""
    if init_logits is not None:
        ws.V.copy_(init_logits)
    elif proposal is not None:
        proposal.propose(ws.V, seed, round_, tau, stream)
    else:
        sat_init_normal(plan, ws.V, seed, round_, init_scale, stream)
    ws.m.zero_()
    ws.v.zero_()
    if steps > 0:
        sat_steps(plan, opt, ws.V, ws.m, ws.v, ws.act, ws.adj, 1, steps, loss=ws.loss, act_dtype=ws.act_dtype,
                  stream=stream, segment=ws.segment)
    sat_threshold(plan, ws.V, ws.bits, ws.keys, stream)
    sat_hard_eval(plan, ws.bits, ws.B, stream)
    sat_cnf_check(plan, ws.bits, ws.valid, ws.B, stream)
    if dedup is not None:
        dedup.insert(ws.keys, ws.valid, ws.B, stream=stream)


def run_epochs(plan: Plan, ws: Workspace, opt: N.OptParams, steps: int, check_every: int, max_age: int, seed: int,
               round_: int, dedup: Dedup, init_scale: float = 1.0, proposal: "Mlp | None" = None, tau: float = 1.0,
               fresh: bool = True, stream=None, events=None):
    """Early exit on device-resident buffers: `steps` descent steps of the batch in
    epochs of `check_every`; after each epoch the valid samples go to `dedup` and
    they (and samples older than max_age) restart (sat_retire, sat_restart) from
    the Philox stream of round round_ + 1 + epoch, or from the proposal.  With
    fresh = False the batch continues from the state of a previous call (V, m, v,
    ws.age) instead of new starts of round round_.  `events` (list): a pair of
    CUDA events recorded around each fused-steps launch is appended.  Returns the
    epochs run."""
    import torch
    if fresh or getattr(ws, "age", None) is None:
        if proposal is not None:
            proposal.propose(ws.V, seed, round_, tau, stream)
        else:
            sat_init_normal(plan, ws.V, seed, round_, init_scale, stream)
        ws.m.zero_()
        ws.v.zero_()
        ws.age = torch.zeros(ws.B, dtype=torch.int32, device=ws.V.device)
        ws.restart = torch.zeros_like(ws.valid)
        ws.src = torch.empty_like(ws.V) if proposal is not None else None
    e, done = 0, 0
    while done < steps:
        kk = min(check_every, steps - done)
        if events is not None:
            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            ev[0].record(stream)
        sat_steps(plan, opt, ws.V, ws.m, ws.v, ws.act, ws.adj, 1, kk, act_dtype=ws.act_dtype, stream=stream,
                  age=ws.age, segment=ws.segment)
        if events is not None:
            ev[1].record(stream)
            events.append((kk, ev))
        sat_threshold(plan, ws.V, ws.bits, ws.keys, stream)
        sat_hard_eval(plan, ws.bits, ws.B, stream)
        sat_cnf_check(plan, ws.bits, ws.valid, ws.B, stream)
        dedup.insert(ws.keys, ws.valid, ws.B, stream=stream)
        sat_retire(ws.valid, ws.age, ws.restart, kk, max_age, ws.B, stream)
        r = round_ + 1 + e
        if proposal is not None:
            if ws.src is None:
                ws.src = torch.empty_like(ws.V)
            proposal.propose(ws.src, seed, r, tau, stream)
        sat_restart(plan, ws.restart, seed, r, ws.V, ws.m, ws.v, init_scale, ws.src, stream)
        done += kk
        e += 1
    return e


def save_checkpoint(path, ws: Workspace, dedup: Dedup | None = None, **meta):
    """Checkpoint of a sampling run between rounds or epochs (numpy .npz): the
    workspace's V, m, v and early-exit ages, the distinct keys found so far, and the
    caller's metadata (for example the next round counter), which load_checkpoint
    returns.  Everything else in a workspace is rewritten before it is read."""
    import json
    import torch
    torch.cuda.synchronize()
    arrays = {"V": ws.V.cpu().numpy(), "m": ws.m.cpu().numpy(), "v": ws.v.cpu().numpy()}
    if ws.age is not None:
        arrays["age"] = ws.age.cpu().numpy()
    if dedup is not None:
        arrays["keys"] = dedup.keys()
    np.savez(path, meta=np.array(json.dumps(meta)), **arrays)


def load_checkpoint(path, ws: Workspace, dedup: Dedup | None = None) -> dict:
    """Restore a save_checkpoint into a workspace of the same plan and batch (and the
    keys into an empty or cleared dedup set, max_batch keys per insert); returns the
    metadata."""
    import json
    import torch
    z = np.load(path)
    for name in ("V", "m", "v"):
        getattr(ws, name).copy_(torch.from_numpy(z[name]))
    if "age" in z.files:
        ws.age = torch.from_numpy(z["age"]).to(ws.V.device)
        ws.restart = torch.zeros_like(ws.valid)
        ws.src = None
    if dedup is not None and "keys" in z.files:
        keys = np.ascontiguousarray(z["keys"]).view(np.int32)
        dedup.clear()
        for i in range(0, len(keys), dedup.max_batch):
            part = torch.from_numpy(keys[i:i + dedup.max_batch]).to(ws.V.device)
            n = part.shape[0]
            words = np.zeros((n + 31) // 32, np.uint32)
            bits = np.packbits(np.ones(n, bool), bitorder="little")
            words.view(np.uint8)[: len(bits)] = bits
            dedup.insert(part, torch.from_numpy(words.view(np.int32)).to(ws.V.device), n)
    torch.cuda.synchronize()
    return json.loads(str(z["meta"]))


def valid_mask(valid_words, B: int) -> np.ndarray:
    w = valid_words.cpu().numpy().view(np.uint32)
    bits = np.unpackbits(w.view(np.uint8), bitorder="little")
    return bits[:B].astype(bool)


def cached_memory() -> tuple[int, int]:
    """(reserved, in use) bytes of the library pool that serves the end-to-end calls'
    workspaces on the current device; the reserve is kept between calls."""
    r, u = C.c_uint64(0), C.c_uint64(0)
    check(lib().sat_cached_memory(C.byref(r), C.byref(u)))
    return r.value, u.value


def release_cached_memory() -> None:
    """Return the library pool's idle reserve on the current device to the device."""
    check(lib().sat_release_cached_memory())


def sample(circuit: Circuit, cnf: Cnf, n_wanted: int, batch=1024, steps=200, max_rounds=1, optimizer="adam",
           lr=0.1, beta1=0.9, beta2=0.999, eps=1e-8, seed=0, first_round=0, init_scale=1.0, act_dtype="f32",
           steps_per_launch=0, proposal: "Mlp | None" = None, tau: float = 1.0, check_every=0, max_age=0,
           recompute_segment=0, step_kernel="auto", stream=None):
    """End to end from host objects (the C call sat_sample); check_every > 0 = early exit;
    recompute_segment > 0 = level-segment recomputation in the fused steps."""
    o = N.SampleOpts()
    lib().sat_sample_opts_default(C.byref(o))
    o.batch, o.steps, o.max_rounds = batch, steps, max_rounds
    o.opt = opt_params(optimizer, lr, beta1, beta2, eps)
    o.seed, o.first_round, o.init_scale = seed, first_round, init_scale
    o.act_dtype, o.steps_per_launch = N.ACT_DTYPES[act_dtype], steps_per_launch
    o.stream = None if stream is None else stream.cuda_stream
    o.proposal = None if proposal is None else proposal.handle
    o.proposal_tau = tau
    o.check_every, o.max_age = check_every, max_age
    o.recompute_segment = recompute_segment
    o.step_kernel = Plan.STEP_KERNELS[step_kernel]
    h = C.c_void_p()
    st = N.SampleStats()
    status = check(lib().sat_sample(circuit.handle, cnf.handle, C.byref(o), n_wanted, C.byref(h), C.byref(st)),
                   allow_partial=True)
    sols = Solutions(h)
    sols.status = status
    sols.stats = _struct_dict(st)
    return sols
