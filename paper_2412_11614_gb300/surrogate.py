"""MLP surrogate of the ISRS EGN integrator: per-channel eta [dB] of a link.

The integrator (egn_nli_eta) supplies the labels.  The network maps per-channel
features to 10 log10(eta): 64 inputs (26 features, zero-padded to the GEMM's
64-wide k blocks) -> 256 -> 256 -> 256 (ReLU) -> 1 (linear).  Weights and
activations are BF16, products accumulate in FP32 on the tensor cores
(egn_mlp_gemm, tcgen05); master weights and Adam state are FP32.  Every step of
training and inference runs in the library's kernels; torch only provides
device memory and streams.

Predictions are only made inside the training envelope (120-channel C+L grid,
identical SSMF spans, N_s, L, Cr and powers within the sampled ranges); other
links are evaluated by the integrator instead.
"""
from __future__ import annotations

import hashlib
import json
import math
import os
from typing import Callable, List, Optional, Sequence

import numpy as np

from . import egn as E
from . import mlp as K

N_FEAT = 26
F_PAD = 64
HIDDEN = 256
LAYERS = 3
C_M_PER_S = 299792458.0


def _moments(fmts):
    m = [E.egn_format_moments(f) for f in fmts]
    return np.array([a for a, _ in m]), np.array([b for _, b in m])


def features(wl) -> np.ndarray:
    """Per-channel feature rows [n_ch][N_FEAT] of a workloads.Workload."""
    f = np.asarray(wl.centre_hz, dtype=np.float64)
    n = len(f)
    fc = 0.5 * (f.min() + f.max())
    x = (f - fc) / 4.5e12
    p_dbm = 10.0 * np.log10(np.asarray(wl.launch_power_w) / 1e-3)
    pm = p_dbm.mean()
    slope = np.polyfit(x, p_dbm, 1)[0] if n > 1 else 0.0
    k = np.ones(9) / 9.0
    local = np.convolve(np.pad(p_dbm, 4, mode="edge"), k, mode="valid")
    phi, psi = _moments(wl.formats)
    local_phi = np.convolve(np.pad(phi, 4, mode="edge"), k, mode="valid")
    s = wl.spans[0]
    ns = len(wl.spans)
    L = s.length_m * 1e-3
    cr = s.cr_per_w_km_thz
    alpha = s.alpha_db_km * math.log(10.0) / 10.0
    leff = (1.0 - math.exp(-alpha * L)) / alpha
    ptot = float(np.sum(wl.launch_power_w))
    btot = (f.max() - f.min()) * 1e-12 * n / max(n - 1, 1)
    drho = cr * ptot * leff * btot  # ISRS tilt scale of Eq. 12 (nepers)
    # interference seen by channel n from channel m scales as (P_m / P_n)^2 and falls
    # with their distance on the grid (cross-channel islands of Eq. 15)
    P = np.asarray(wl.launch_power_w, dtype=np.float64)
    dist = np.abs(np.arange(n)[:, None] - np.arange(n)[None, :]).astype(np.float64)
    off = dist > 0
    k1 = np.where(off, 1.0 / np.where(off, dist, 1.0), 0.0)
    k2 = k1 * k1
    p2 = P * P
    x1 = (k1 @ p2) / (p2 + 1e-300)
    x2 = (k2 @ p2) / (p2 + 1e-300)
    phi_w = (k1 @ (phi * p2)) / np.maximum(k1 @ p2, 1e-300)
    edge = np.minimum(np.arange(n), n - 1 - np.arange(n)) / max(n / 2.0, 1.0)
    cols = [x, x ** 2, x ** 3, (p_dbm - 1.0) / 3.0, np.full(n, (pm - 1.0) / 3.0), np.full(n, slope / 3.0),
            (local - pm) / 2.0, np.full(n, (cr - 0.028) / 0.014), np.full(n, (L - 85.0) / 35.0),
            np.full(n, (ns - 15.5) / 15.0), np.full(n, math.log(ns) / math.log(30.0)), phi, psi / 10.0,
            np.full(n, phi.mean()), local_phi, np.full(n, 1.0 / ns), np.full(n, drho), np.ones(n),
            np.log10(np.maximum(x1, 1e-300)) / 2.0, np.log10(np.maximum(x2, 1e-300)) / 2.0, phi_w, edge,
            np.full(n, ns * L / 3000.0), np.full(n, math.log(leff)), np.full(n, math.log(ns) * math.log(L / 85.0)),
            np.full(n, math.log(ns) ** 2 / 10.0)]
    return np.stack(cols, axis=1).astype(np.float64)


def in_envelope(wl, n_ch: int = 120) -> bool:
    """True if the link is of the kind the surrogates were trained on: the n_ch
    channel 64 GBd grid of the seeded training links, identical SSMF spans, N_s,
    L, Cr and powers inside the sampled ranges."""
    if len(wl.centre_hz) != n_ch or any(r != 64e9 for r in wl.symbol_rate_baud):
        return False
    s0 = wl.spans[0]
    if any(s != s0 for s in wl.spans):
        return False
    ns, L, cr = len(wl.spans), s0.length_m * 1e-3, s0.cr_per_w_km_thz
    p = 10.0 * np.log10(np.asarray(wl.launch_power_w) / 1e-3)
    return (1 <= ns <= 30 and 50.0 <= L <= 120.0 and 0.014 <= cr <= 0.042 and abs(s0.D_ps_nm_km - 17.0) < 1e-9
            and -6.0 <= p.min() and p.max() <= 8.0)


class Surrogate:
    """The MLP with its device state (torch tensors as device memory)."""

    def __init__(self, seed: int = 0, device: str = "cuda"):
        import torch
        self.torch = torch
        self.dev = device
        rng = np.random.default_rng(seed)
        dims = [F_PAD] + [HIDDEN] * LAYERS
        self.W, self.b, self.Wb, self.WbT = [], [], [], []
        # weights and biases uniform in +-1/sqrt(fan_in) (on these labels it generalises
        # better than a He-normal start with zero biases)
        for i in range(LAYERS):
            fan_in = N_FEAT if i == 0 else dims[i]
            lim = 1.0 / math.sqrt(fan_in)
            w = np.zeros((dims[i + 1], dims[i]), dtype=np.float32)
            w[:, :fan_in] = rng.uniform(-lim, lim, size=(dims[i + 1], fan_in))
            self.W.append(torch.tensor(w, device=device))
            self.b.append(torch.tensor(rng.uniform(-lim, lim, dims[i + 1]).astype(np.float32), device=device))
            self.Wb.append(torch.empty(w.shape, dtype=torch.bfloat16, device=device))
            self.WbT.append(torch.empty((w.shape[1], w.shape[0]), dtype=torch.bfloat16, device=device))
        lim = 1.0 / math.sqrt(HIDDEN)
        self.w_out = torch.tensor(rng.uniform(-lim, lim, HIDDEN).astype(np.float32), device=device)
        self.b_out = torch.tensor(rng.uniform(-lim, lim, 1).astype(np.float32), device=device)
        self.params = [p for pair in zip(self.W, self.b) for p in pair] + [self.w_out, self.b_out]
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.step_count = 0
        self.err = torch.zeros(1, dtype=torch.int32, device=device)
        self.x_mean = np.zeros(N_FEAT)
        self.x_std = np.ones(N_FEAT)
        self.y_mean, self.y_std = 0.0, 1.0
        self._refresh_bf16(None)

    # ------------------------------------------------------------------ helpers
    def _refresh_bf16(self, stream):
        for i in range(LAYERS):
            K.cast(self.W[i], self.Wb[i], stream=stream)
            K.transpose(self.Wb[i], self.Wb[i].shape[0], self.WbT[i], stream=stream)

    def _buffers(self, rows_pad):
        torch = self.torch
        if getattr(self, "_rows", None) == rows_pad:
            return
        self._rows = rows_pad
        bf = torch.bfloat16
        self.h = [torch.zeros((rows_pad, F_PAD), dtype=bf, device=self.dev)] + \
                 [torch.empty((rows_pad, HIDDEN), dtype=bf, device=self.dev) for _ in range(LAYERS)]
        self.y = torch.empty(rows_pad, dtype=torch.float32, device=self.dev)
        self.g = torch.empty(rows_pad, dtype=torch.float32, device=self.dev)
        self.loss = torch.empty(1, dtype=torch.float32, device=self.dev)
        self.dh = [torch.empty((rows_pad, HIDDEN), dtype=bf, device=self.dev) for _ in range(2)]
        self.dhT = torch.empty((HIDDEN, rows_pad), dtype=bf, device=self.dev)
        self.hT = torch.empty((HIDDEN, rows_pad), dtype=bf, device=self.dev)
        kb = rows_pad // 64                   # 64-row k blocks of the weight-gradient GEMMs
        per = -(-kb // 16)                    # at most 16 k splits, none empty
        self.splits = -(-kb // per)
        self.part = torch.empty(self.splits * HIDDEN * HIDDEN, dtype=torch.float32, device=self.dev)
        self.grads = [torch.empty_like(p) for p in self.params]
        self.xf = torch.empty((rows_pad, F_PAD), dtype=torch.float32, device=self.dev)

    def _load_inputs(self, x: np.ndarray, stream):
        """Normalised features (host FP32) -> BF16 input rows on the device."""
        torch = self.torch
        rows = x.shape[0]
        rows_pad = ((rows + 63) // 64) * 64
        self._buffers(rows_pad)
        xp = np.zeros((rows_pad, F_PAD), dtype=np.float32)
        xp[:rows, :N_FEAT] = (x - self.x_mean) / self.x_std
        self.xf.copy_(torch.from_numpy(xp), non_blocking=False)
        K.cast(self.xf, self.h[0], stream=stream)
        return rows, rows_pad

    def _forward(self, stream):
        for i in range(LAYERS):
            K.gemm(self.h[i], self.Wb[i], self.h[i + 1], K.EPI_BIAS_RELU, bias=self.b[i], err=self.err, stream=stream)

    # ------------------------------------------------------------------ API
    def predict_rows(self, x: np.ndarray, stream=None) -> np.ndarray:
        """Predicted 10 log10(eta) for feature rows x [rows][N_FEAT]."""
        rows, _ = self._load_inputs(x, stream)
        self._forward(stream)
        K.head(self.h[LAYERS], self.w_out, self.b_out, self.y, stream=stream)
        self._check()
        return self.y[:rows].cpu().numpy() * self.y_std + self.y_mean

    def train_step(self, x: np.ndarray, t: np.ndarray, lr: float, stream=None) -> float:
        """One Adam step on feature rows x and targets t (10 log10 eta)."""
        torch = self.torch
        rows, rows_pad = self._load_inputs(x, stream)
        tn = np.zeros(rows_pad, dtype=np.float32)
        tn[:rows] = (t - self.y_mean) / self.y_std
        mask = np.zeros(rows_pad, dtype=np.float32)
        mask[:rows] = 1.0
        tgt = torch.from_numpy(tn).to(self.dev)
        msk = torch.from_numpy(mask).to(self.dev)
        self._forward(stream)
        gw_out, gb_out = self.grads[-2], self.grads[-1]
        K.head(self.h[LAYERS], self.w_out, self.b_out, self.y, target=tgt, mask=msk, loss=self.loss, g=self.g,
               dh=self.dh[0], dw=gw_out, db=gb_out, stream=stream)
        cur = 0
        for i in reversed(range(LAYERS)):
            dh = self.dh[cur]
            fan = self.h[i].shape[1]
            # weight gradient dW_i = dh^T h_i (k = rows, split over CTA layers), bias gradient
            K.transpose(dh, rows_pad, self.dhT, stream=stream)
            hT = self.hT[:fan]
            K.transpose(self.h[i], rows_pad, hT, stream=stream)
            part = self.part[: self.splits * HIDDEN * fan]  # dense [splits][HIDDEN][fan]
            K.gemm(self.dhT, hT, part, K.EPI_F32, splits=self.splits, err=self.err, stream=stream)
            K.reduce_splits(part, self.splits, self.grads[2 * i], stream=stream)
            K.colsum(dh, self.grads[2 * i + 1], stream=stream)
            if i > 0:  # gradient of the layer below, through its ReLU
                K.gemm(dh, self.WbT[i], self.dh[1 - cur], K.EPI_RELU_GRAD, aux=self.h[i], err=self.err,
                       stream=stream)
                cur = 1 - cur
        self.step_count += 1
        for p, g, m, v in zip(self.params, self.grads, self.m, self.v):
            K.adam(p, g, m, v, lr, self.step_count, stream=stream)
        self._refresh_bf16(stream)
        self._check()
        return float(self.loss.item())

    def _check(self):
        e = int(self.err.item())
        if e:
            raise RuntimeError(f"a tensor-core kernel's bounded wait ran out (code {e})")

    def fit_normalisation(self, x: np.ndarray, t: np.ndarray):
        self.x_mean = x.mean(axis=0)
        self.x_std = np.where(x.std(axis=0) > 1e-12, x.std(axis=0), 1.0)
        self.y_mean, self.y_std = float(t.mean()), float(t.std() or 1.0)

    # ------------------------------------------------------------------ checkpoints
    def state(self) -> dict:
        """Host copy of everything training needs to continue: FP32 master
        weights, Adam moments, step count and the normalisation."""
        st = {"step_count": np.int64(self.step_count), "x_mean": self.x_mean, "x_std": self.x_std,
              "y_norm": np.array([self.y_mean, self.y_std])}
        for j, (p, m, v) in enumerate(zip(self.params, self.m, self.v)):
            st[f"p{j}"] = p.cpu().numpy()
            st[f"m{j}"] = m.cpu().numpy()
            st[f"v{j}"] = v.cpu().numpy()
        return st

    def load_state(self, st) -> None:
        torch = self.torch
        for j, (p, m, v) in enumerate(zip(self.params, self.m, self.v)):
            for dst, key in ((p, f"p{j}"), (m, f"m{j}"), (v, f"v{j}")):
                src = np.asarray(st[key])
                if src.shape != tuple(dst.shape):
                    raise ValueError(f"checkpoint {key}: shape {src.shape}, model {tuple(dst.shape)}")
                dst.copy_(torch.from_numpy(src))
        self.step_count = int(st["step_count"])
        self.x_mean, self.x_std = np.asarray(st["x_mean"]), np.asarray(st["x_std"])
        self.y_mean, self.y_std = (float(a) for a in np.asarray(st["y_norm"]))
        self._refresh_bf16(None)


# --------------------------------------------------------------------------- per-link network

LINK_HIDDEN = 512
LINK_LAYERS = 3


def _pad64(n: int) -> int:
    return -(-n // 64) * 64


def link_features(wl) -> np.ndarray:
    """One input row per link: the n_ch launch powers [dBm], the span count, the
    span length [km] and Cr [1/(W km THz)] (n_ch + 3 values)."""
    s = wl.spans[0]
    p_dbm = 10.0 * np.log10(np.asarray(wl.launch_power_w) / 1e-3)
    return np.concatenate([p_dbm, [len(wl.spans), s.length_m * 1e-3, s.cr_per_w_km_thz]]).astype(np.float64)


class LinkSurrogate:
    """The network that maps a whole link to all its channels at once: n_ch
    launch powers + span count + span length + Cr -> 3 x 512 GELU -> n_ch values
    of 10 log10(eta).  Inputs are zero-padded to a multiple of 64 (the GEMM's k
    blocks), the output layer to a multiple of 64 rows.  BF16 weights and
    activations on the tensor cores (egn_mlp_gemm with the GELU epilogues, the
    pre-activations kept in BF16 for the backward pass), FP32 output layer and
    loss (egn_mlp_outputs), FP32 masters and Adam.  The same train() and
    checkpoints as Surrogate; targets are [links][n_ch] arrays."""

    def __init__(self, n_ch: int = 120, seed: int = 0, device: str = "cuda"):
        import torch
        self.torch = torch
        self.dev = device
        self.n_ch = n_ch
        self.n_in = n_ch + 3
        self.in_pad = _pad64(self.n_in)
        self.out_pad = _pad64(n_ch)
        rng = np.random.default_rng(seed)
        dims = [self.in_pad] + [LINK_HIDDEN] * LINK_LAYERS
        self.W, self.b, self.Wb, self.WbT = [], [], [], []
        for i in range(LINK_LAYERS):
            fan_in = self.n_in if i == 0 else dims[i]
            lim = 1.0 / math.sqrt(fan_in)
            w = np.zeros((dims[i + 1], dims[i]), dtype=np.float32)
            w[:, :fan_in] = rng.uniform(-lim, lim, size=(dims[i + 1], fan_in))
            self.W.append(torch.tensor(w, device=device))
            self.b.append(torch.tensor(rng.uniform(-lim, lim, dims[i + 1]).astype(np.float32), device=device))
            self.Wb.append(torch.empty(w.shape, dtype=torch.bfloat16, device=device))
            self.WbT.append(torch.empty((w.shape[1], w.shape[0]), dtype=torch.bfloat16, device=device))
        lim = 1.0 / math.sqrt(LINK_HIDDEN)
        wo = np.zeros((self.out_pad, LINK_HIDDEN), dtype=np.float32)
        wo[:n_ch] = rng.uniform(-lim, lim, size=(n_ch, LINK_HIDDEN))
        self.w_out = torch.tensor(wo, device=device)
        self.b_out = torch.tensor(rng.uniform(-lim, lim, n_ch).astype(np.float32), device=device)
        self.wb_out = torch.empty(wo.shape, dtype=torch.bfloat16, device=device)
        self.wb_outT = torch.empty((LINK_HIDDEN, self.out_pad), dtype=torch.bfloat16, device=device)
        self.params = [p for pair in zip(self.W, self.b) for p in pair] + [self.w_out, self.b_out]
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.step_count = 0
        self.err = torch.zeros(1, dtype=torch.int32, device=device)
        self.x_mean = np.zeros(self.n_in)
        self.x_std = np.ones(self.n_in)
        self.y_mean, self.y_std = np.zeros(n_ch), np.ones(n_ch)
        self._refresh_bf16(None)

    def _refresh_bf16(self, stream):
        for i in range(LINK_LAYERS):
            K.cast(self.W[i], self.Wb[i], stream=stream)
            K.transpose(self.Wb[i], self.Wb[i].shape[0], self.WbT[i], stream=stream)
        K.cast(self.w_out, self.wb_out, stream=stream)
        K.transpose(self.wb_out, self.out_pad, self.wb_outT, stream=stream)

    def _buffers(self, rows_pad):
        torch = self.torch
        if getattr(self, "_rows", None) == rows_pad:
            return
        self._rows = rows_pad
        bf, H = torch.bfloat16, LINK_HIDDEN
        self.h = [torch.zeros((rows_pad, self.in_pad), dtype=bf, device=self.dev)] + \
                 [torch.empty((rows_pad, H), dtype=bf, device=self.dev) for _ in range(LINK_LAYERS)]
        self.z = [None] + [torch.empty((rows_pad, H), dtype=bf, device=self.dev) for _ in range(LINK_LAYERS)]
        self.acc = torch.empty((rows_pad, self.out_pad), dtype=torch.float32, device=self.dev)
        self.y = torch.empty((rows_pad, self.n_ch), dtype=torch.float32, device=self.dev)
        self.loss = torch.empty(1, dtype=torch.float32, device=self.dev)
        self.g = torch.empty((rows_pad, self.out_pad), dtype=bf, device=self.dev)
        self.gT = torch.empty((self.out_pad, rows_pad), dtype=bf, device=self.dev)
        self.dz = [torch.empty((rows_pad, H), dtype=bf, device=self.dev) for _ in range(2)]
        self.dzT = torch.empty((H, rows_pad), dtype=bf, device=self.dev)
        self.hT = torch.empty((max(H, self.in_pad), rows_pad), dtype=bf, device=self.dev)
        kb = rows_pad // 64
        per = -(-kb // 16)
        self.splits = -(-kb // per)
        self.part = torch.empty(self.splits * max(H, self.out_pad) * max(H, self.in_pad), dtype=torch.float32,
                                device=self.dev)
        self.grads = [torch.empty_like(p) for p in self.params]
        self.xf = torch.empty((rows_pad, self.in_pad), dtype=torch.float32, device=self.dev)

    def _load_inputs(self, x: np.ndarray, stream):
        torch = self.torch
        rows = x.shape[0]
        rows_pad = ((rows + 63) // 64) * 64
        self._buffers(rows_pad)
        xp = np.zeros((rows_pad, self.in_pad), dtype=np.float32)
        xp[:rows, :self.n_in] = (x - self.x_mean) / self.x_std
        self.xf.copy_(torch.from_numpy(xp))
        K.cast(self.xf, self.h[0], stream=stream)
        return rows, rows_pad

    def _forward(self, rows, rows_pad, stream):
        for i in range(LINK_LAYERS):
            K.gemm(self.h[i], self.Wb[i], self.h[i + 1], K.EPI_BIAS_GELU, bias=self.b[i], aux=self.z[i + 1],
                   err=self.err, stream=stream)
        K.gemm(self.h[LINK_LAYERS], self.wb_out, self.acc, K.EPI_F32, err=self.err, stream=stream)

    def predict_rows(self, x: np.ndarray, stream=None) -> np.ndarray:
        """10 log10(eta) [links][n_ch] for input rows x [links][n_ch + 3]."""
        rows, rows_pad = self._load_inputs(np.atleast_2d(x), stream)
        self._forward(rows, rows_pad, stream)
        K.outputs(self.acc, rows, rows_pad, self.n_ch, self.b_out, self.y, stream=stream)
        self._check()
        return self.y[:rows].cpu().numpy().astype(np.float64) * self.y_std + self.y_mean

    def train_step(self, x: np.ndarray, t: np.ndarray, lr: float, stream=None) -> float:
        """One Adam step on input rows x [links][n_ch + 3] and targets t [links][n_ch]."""
        torch = self.torch
        rows, rows_pad = self._load_inputs(x, stream)
        tn = np.zeros((rows_pad, self.n_ch), dtype=np.float32)
        tn[:rows] = (t - self.y_mean) / self.y_std
        mask = np.zeros(rows_pad, dtype=np.float32)
        mask[:rows] = 1.0
        tgt = torch.from_numpy(tn).to(self.dev)
        msk = torch.from_numpy(mask).to(self.dev)
        self._forward(rows, rows_pad, stream)
        H = LINK_HIDDEN
        K.outputs(self.acc, rows_pad, rows_pad, self.n_ch, self.b_out, self.y, target=tgt, mask=msk, loss=self.loss,
                  g=self.g, db=self.grads[-1], stream=stream)
        # output layer: dW_out = g^T h3 (k = rows), dz3 = (g W_out) GELU'(z3)
        K.transpose(self.g, rows_pad, self.gT, stream=stream)
        hT = self.hT[:H]
        K.transpose(self.h[LINK_LAYERS], rows_pad, hT, stream=stream)
        part = self.part[: self.splits * self.out_pad * H]
        K.gemm(self.gT, hT, part, K.EPI_F32, splits=self.splits, err=self.err, stream=stream)
        K.reduce_splits(part, self.splits, self.grads[-2], stream=stream)
        cur = 0
        K.gemm(self.g, self.wb_outT, self.dz[cur], K.EPI_GELU_GRAD, aux=self.z[LINK_LAYERS], err=self.err,
               stream=stream)
        for i in reversed(range(LINK_LAYERS)):  # layer i maps h[i] to z[i + 1]
            dz = self.dz[cur]
            fan = self.h[i].shape[1]
            K.transpose(dz, rows_pad, self.dzT, stream=stream)
            hT = self.hT[:fan]
            K.transpose(self.h[i], rows_pad, hT, stream=stream)
            part = self.part[: self.splits * H * fan]
            K.gemm(self.dzT, hT, part, K.EPI_F32, splits=self.splits, err=self.err, stream=stream)
            K.reduce_splits(part, self.splits, self.grads[2 * i], stream=stream)
            K.colsum(dz, self.grads[2 * i + 1], stream=stream)
            if i > 0:
                K.gemm(dz, self.WbT[i], self.dz[1 - cur], K.EPI_GELU_GRAD, aux=self.z[i], err=self.err, stream=stream)
                cur = 1 - cur
        self.step_count += 1
        for p, g, m, v in zip(self.params, self.grads, self.m, self.v):
            K.adam(p, g, m, v, lr, self.step_count, stream=stream)
        self._refresh_bf16(stream)
        self._check()
        return float(self.loss.item())

    def _check(self):
        e = int(self.err.item())
        if e:
            raise RuntimeError(f"a tensor-core kernel's bounded wait ran out (code {e})")

    def fit_normalisation(self, x: np.ndarray, t: np.ndarray):
        self.x_mean = x.mean(axis=0)
        sd = x.std(axis=0)
        self.x_std = np.where(sd > 1e-12, sd, 1.0)
        self.y_mean = t.mean(axis=0)
        sd = t.std(axis=0)
        self.y_std = np.where(sd > 1e-12, sd, 1.0)

    def state(self) -> dict:
        st = {"step_count": np.int64(self.step_count), "x_mean": self.x_mean, "x_std": self.x_std,
              "y_mean": self.y_mean, "y_std": self.y_std}
        for j, (p, m, v) in enumerate(zip(self.params, self.m, self.v)):
            st[f"p{j}"] = p.cpu().numpy()
            st[f"m{j}"] = m.cpu().numpy()
            st[f"v{j}"] = v.cpu().numpy()
        return st

    def load_state(self, st) -> None:
        torch = self.torch
        for j, (p, m, v) in enumerate(zip(self.params, self.m, self.v)):
            for dst, key in ((p, f"p{j}"), (m, f"m{j}"), (v, f"v{j}")):
                src = np.asarray(st[key])
                if src.shape != tuple(dst.shape):
                    raise ValueError(f"checkpoint {key}: shape {src.shape}, model {tuple(dst.shape)}")
                dst.copy_(torch.from_numpy(src))
        self.step_count = int(st["step_count"])
        self.x_mean, self.x_std = np.asarray(st["x_mean"]), np.asarray(st["x_std"])
        self.y_mean, self.y_std = np.asarray(st["y_mean"]), np.asarray(st["y_std"])
        self._refresh_bf16(None)


def _save_atomic(path: str, arrays: dict) -> None:
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        np.savez(f, **arrays)
    os.replace(tmp, path)


def train(model: Surrogate, x: np.ndarray, t: np.ndarray, steps: int, batch_rows: int = 8192,
          lr_max: float = 2e-3, lr_min: float = 1e-5, seed: int = 0, checkpoint: Optional[str] = None,
          every: int = 0, on_step: Optional[Callable[[int, float], None]] = None) -> List[float]:
    """Adam on minibatches of rows (a fresh permutation every epoch, cosine
    learning rate from lr_max to lr_min).  With `checkpoint`, the model, the
    sampler's state and the step are saved there every `every` steps and at the
    end, and a run that finds the file continues from it: the result is bit for
    bit that of an uninterrupted run.  Returns the losses of the steps run here."""
    rng = np.random.default_rng(seed)
    per_epoch = max(1, len(x) // batch_rows)
    perm = None
    start = 0
    if checkpoint and os.path.exists(checkpoint):
        with np.load(checkpoint, allow_pickle=False) as z:
            model.load_state(z)
            start = int(z["next_step"])
            rng.bit_generator.state = json.loads(str(z["rng"]))
            perm = z["perm"] if z["perm"].size else None
    losses = []

    def save(next_step):
        st = model.state()
        st.update(next_step=np.int64(next_step), rng=np.array(json.dumps(rng.bit_generator.state)),
                  perm=perm if perm is not None else np.zeros(0, dtype=np.int64))
        _save_atomic(checkpoint, st)

    for step in range(start, steps):
        if step % per_epoch == 0:
            perm = rng.permutation(len(x))
        j = (step % per_epoch) * batch_rows
        idx = perm[j:j + batch_rows]
        lr = lr_min + 0.5 * (lr_max - lr_min) * (1 + math.cos(math.pi * step / steps))
        loss = model.train_step(x[idx], t[idx], lr)
        losses.append(loss)
        if checkpoint and every and (step + 1) % every == 0:
            save(step + 1)
        if on_step:
            on_step(step, loss)
    if checkpoint and start < steps:
        save(steps)
    return losses


def labels(workloads: Sequence, opts, rule: int = E.EGN_RULE_GL) -> List[np.ndarray]:
    """10 log10(eta) of every channel of every link, from the integrator (one
    batch evaluation) with the node rule `rule` (EGN_RULE_RIDGE: the
    ridge-resolving rule, opts.gl_order nodes per piece, n_min 4)."""
    links = [E.link_from_workload(w) for w in workloads]
    if rule != E.EGN_RULE_GL:
        for ln in links:
            ln.set_node_rule(rule, 4)
    out = E.nli_eta_batch(links, opts)
    for ln in links:
        ln.close()
    return [10.0 * np.log10(e) for e, _ in out]


def generate_labels(directory: str, seeds: Sequence[int], opts, shard_links: int = 256,
                    label_fn: Optional[Callable] = None, make_link: Optional[Callable] = None,
                    rule: int = E.EGN_RULE_GL) -> np.ndarray:
    """Labels of the seeded links, written shard by shard under `directory`.

    shard_NNNNN.npy holds the [links][channels] float64 array of 10 log10 eta for
    seeds[k * shard_links : (k + 1) * shard_links]; index.json records the run
    (a hash of the seed list, the options, the shard size) and the shards that
    are complete.  A shard file is written first and entered in the index after,
    both by atomic rename, so a run that is killed loses at most the shard in
    progress and a rerun with the same arguments computes only the shards the
    index does not list.  Files of a different run (other seeds or options) are
    refused.  label_fn(workloads) -> list of per-channel arrays (default: the
    integrator with node rule `rule`, batches of 64 links); make_link(seed) ->
    workload (default: the seeded 120-channel training links).  Returns all
    labels, [links][channels]."""
    if make_link is None:
        from .workloads import surrogate_link as make_link
    if label_fn is None:
        def label_fn(wls):
            out = []
            for i in range(0, len(wls), 64):
                out += labels(wls[i:i + 64], opts, rule)
            return out
    seeds = [int(s) for s in seeds]
    key = {"seeds_sha256": hashlib.sha256(np.asarray(seeds, dtype=np.int64).tobytes()).hexdigest(),
           "n_links": len(seeds), "shard_links": int(shard_links),
           "opts": {f: getattr(opts, f) for f in ("gl_order", "dz_km", "mu_form", "precision", "terms")}
           if opts is not None else None}
    if rule != E.EGN_RULE_GL:  # runs of the configured rule keep their earlier keys
        key["rule"] = int(rule)
    os.makedirs(directory, exist_ok=True)
    index_path = os.path.join(directory, "index.json")
    done = set()
    if os.path.exists(index_path):
        with open(index_path) as f:
            idx = json.load(f)
        if idx.get("run") != key:
            raise ValueError(f"{directory} holds labels of another run: {idx.get('run')} != {key}")
        done = set(idx["done"])
    n_shards = -(-len(seeds) // shard_links)
    for k in range(n_shards):
        if k in done:
            continue
        part = seeds[k * shard_links:(k + 1) * shard_links]
        lab = np.asarray(label_fn([make_link(s) for s in part]), dtype=np.float64)
        shard = os.path.join(directory, f"shard_{k:05d}.npy")
        with open(shard + ".tmp", "wb") as f:
            np.save(f, lab)
        os.replace(shard + ".tmp", shard)
        done.add(k)
        with open(index_path + ".tmp", "w") as f:
            json.dump({"run": key, "done": sorted(done)}, f)
        os.replace(index_path + ".tmp", index_path)
    return np.concatenate([np.load(os.path.join(directory, f"shard_{k:05d}.npy")) for k in range(n_shards)])


def predict(model, workloads: Sequence, opts, n_ch: int = 120, rule: int = E.EGN_RULE_GL):
    """10 log10(eta) per link: the network inside the training envelope, the
    integrator outside it (node rule `rule`, as the labels).  `model` is a
    Surrogate (per-channel rows) or a LinkSurrogate (one row per link).  Returns
    (list of arrays, list of bools: used the network)."""
    inside = [in_envelope(w, n_ch) for w in workloads]
    res: List = [None] * len(workloads)
    idx = [i for i, ok in enumerate(inside) if ok]
    if idx and isinstance(model, LinkSurrogate):
        y = model.predict_rows(np.stack([link_features(workloads[i]) for i in idx]))
        for k, i in enumerate(idx):
            res[i] = y[k]
    elif idx:
        x = np.concatenate([features(workloads[i]) for i in idx])
        y = model.predict_rows(x)
        o = 0
        for i in idx:
            n = len(workloads[i].centre_hz)
            res[i] = y[o:o + n]
            o += n
    rest = [i for i, ok in enumerate(inside) if not ok]
    if rest:
        for i, lab in zip(rest, labels([workloads[i] for i in rest], opts, rule)):
            res[i] = lab
    return res, inside
