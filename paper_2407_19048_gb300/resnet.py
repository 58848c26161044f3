"""ResNet-1D data summary (Sec. 4): the paper's embedding network on the whitened strain.

A stem convolution (kernel 7, stride 2, 64 channels), group normalisation, ReLU and a
max pool, then stacks of basic residual blocks with 64, 128 and 256 channels ((5, 3, 3)
blocks, kernel 5, the first block of a stack striding by 2 with a 1 x 1 projection on
the shortcut), the mean over time and a fully connected layer to the representation.
The stride-1 kernel-5 convolutions are implicit GEMMs on the tensor cores
(`gwx_conv1d_bf16`: the A tiles come from a 3-D tensor map of the activations; backward
`gwx_conv1d_bf16_backward`: the input gradient is the same product with mirrored taps, the
weight gradient a split-K product over transposed rows); the stem, the strided entries and
the 1 x 1 shortcuts use im2col rows times the weights (`gwx_im2col`, `gwx_dense_bf16`;
backward `gwx_dense_bf16_backward`, `gwx_col2im`).  Normalisation, residual addition and
ReLU are fused (`gwx_group_norm`), and the backward pass mirrors the forward call by call.
Activations are channels-last bfloat16, convolution outputs FP32.
"""
import ctypes
import math

from . import _lib

STAGES = ((64, 5, 1), (128, 3, 2), (256, 3, 2))
GROUPS = 8


def stem_k(D):
    return (7 * D + 7) // 8 * 8


class ResNet1D:
    def __init__(self, D, out_dim, stages=STAGES, device=None, seed=0, params=None, implicit=True):
        """implicit: run the stride-1 kernel-5 convolutions whose channel counts are
        multiples of 64 and whose series are multiples of 128 steps as implicit GEMMs
        (gwx_conv1d_bf16: no im2col rows, the input gradient without col2im); the others
        (stem, strided entries, 1 x 1 shortcuts) always use im2col rows."""
        import torch
        import paper_2407_19048_gb300 as gwx
        self.gwx = gwx
        self.implicit = bool(implicit)
        self.dev = device or torch.device("cuda", torch.cuda.current_device())
        self.D, self.out_dim, self.stages = D, out_dim, tuple(stages)
        if params is None:
            import numpy as np
            params = self._init(np.random.default_rng(seed))
        self.load(params)

    # ------------------------------------------------------------------ parameters
    def _init(self, rng):
        """Weights N(0, 2 / fan_in), group-norm scale 1 and shift 0, FC N(0, 1 / fan_in)."""
        import numpy as np

        def w(o, i):
            return rng.normal(0, math.sqrt(2.0 / i), (o, i))

        c0 = self.stages[0][0]
        P = {"W0": np.zeros((c0, stem_k(self.D))), "g0": np.ones(c0), "b0": np.zeros(c0)}
        P["W0"][:, :7 * self.D] = w(c0, 7 * self.D)
        cin, blocks = c0, []
        for (c, n, s) in self.stages:
            for i in range(n):
                stride = s if i == 0 else 1
                blk = {"s": stride, "W1": w(c, 5 * cin), "W2": w(c, 5 * c), "g1": np.ones(c), "b1": np.zeros(c),
                       "g2": np.ones(c), "b2": np.zeros(c)}
                if stride != 1 or cin != c:
                    blk.update(Wd=w(c, cin), gd=np.ones(c), bd=np.zeros(c))
                blocks.append(blk)
                cin = c
        P["blocks"] = blocks
        P["Wf"] = rng.normal(0, math.sqrt(1.0 / cin), (self.out_dim, cin))
        P["bf"] = np.zeros(self.out_dim)
        return P

    def load(self, P):
        """Parameters from a dict of arrays (the layout of oracle.resnet.init_params)."""
        import torch

        def t(a):
            return torch.as_tensor(a, dtype=torch.float32, device=self.dev).contiguous()

        self.P = {k: t(v) for k, v in P.items() if k != "blocks"}
        self.blocks = []
        for blk in P["blocks"]:
            self.blocks.append({k: (v if k == "s" else t(v)) for k, v in blk.items()})
        self.refresh()

    def refresh(self):
        """bfloat16 copies of the convolution and FC weights."""
        import torch
        self.W16 = {k: self.P[k].to(torch.bfloat16) for k in ("W0", "Wf")}
        for blk in self.blocks:
            for k in ("W1", "W2", "Wd"):
                if k in blk:
                    blk[k + "16"] = blk[k].to(torch.bfloat16)

    def tensors(self):
        """(name, FP32 tensor, bfloat16 copy or None) of every trainable tensor."""
        out = [("W0", self.P["W0"], self.W16["W0"]), ("g0", self.P["g0"], None), ("b0", self.P["b0"], None)]
        for i, blk in enumerate(self.blocks):
            for k in ("W1", "g1", "b1", "W2", "g2", "b2", "Wd", "gd", "bd"):
                if k in blk:
                    out.append(("%d.%s" % (i, k), blk[k], blk.get(k + "16")))
        out += [("Wf", self.P["Wf"], self.W16["Wf"]), ("bf", self.P["bf"], None)]
        return out

    # ------------------------------------------------------------------ pieces
    def _implicit_ok(self, x, W16, k, s, cf):
        if not self.implicit or cf or s != 1 or k != 5:
            return False
        _, T, C = x.shape
        return T % 128 == 0 and C % 64 == 0 and W16.shape[0] % 64 == 0

    def _conv(self, x, W16, k, s, p, cf=False):
        """(z [B][T_out][C_out] FP32, cols) of bfloat16 x [B][T][C] (cf: FP32 [B][D][N]);
        cols is None when the convolution ran as an implicit GEMM."""
        import torch
        gwx, lib = self.gwx, _lib.load()
        if self._implicit_ok(x, W16, k, s, cf):
            return gwx.conv1d_bf16(x, W16, k), None
        st = gwx._stream()
        K = W16.shape[1]
        if cf:
            B, C, T = x.shape
        else:
            B, T, C = x.shape
        To = (T + 2 * p - k) // s + 1
        cols = torch.empty((B * To, K), dtype=torch.bfloat16, device=self.dev)
        if cf:
            gwx._check(lib.gwx_im2col_cf(gwx._ptr(x), B, C, T, k, s, p, K, gwx._ptr(cols), st))
        else:
            gwx._check(lib.gwx_im2col(gwx._ptr(x), B, T, C, k, s, p, K, gwx._ptr(cols), st))
        z = gwx.dense_bf16(cols, W16, None, act=gwx.ACT_NONE, out_dtype=torch.float32)
        return z.view(B, To, -1), cols

    def _gn(self, z, g, b, relu, res32=None, res16=None, out32=False):
        import torch
        gwx, lib = self.gwx, _lib.load()
        B, T, C = z.shape
        ms = torch.empty((B, GROUPS, 2), dtype=torch.float32, device=self.dev)
        o16 = None if out32 else torch.empty((B, T, C), dtype=torch.bfloat16, device=self.dev)
        o32 = torch.empty((B, T, C), dtype=torch.float32, device=self.dev) if out32 else None
        gwx._check(lib.gwx_group_norm(gwx._ptr(z), B, T, C, GROUPS, gwx._ptr(g), gwx._ptr(b),
                                      gwx._ptr(res32) if res32 is not None else None,
                                      gwx._ptr(res16) if res16 is not None else None, 1 if relu else 0,
                                      gwx._ptr(o16) if o16 is not None else None,
                                      gwx._ptr(o32) if o32 is not None else None, gwx._ptr(ms), gwx._stream()))
        return (o32 if out32 else o16), ms

    # ------------------------------------------------------------------ forward / backward
    def forward(self, y, out_dtype=None):
        """Representation [B][out_dim] (FP32, or out_dtype) of whitened windows y [B][D][N]
        (FP32)."""
        import torch
        gwx, lib = self.gwx, _lib.load()
        st = gwx._stream()
        tape = {}
        z0, cols0 = self._conv(y, self.W16["W0"], 7, 2, 3, cf=True)
        a0, ms0 = self._gn(z0, self.P["g0"], self.P["b0"], True)
        B, T1, C0 = a0.shape
        To = (T1 + 2 - 3) // 2 + 1
        h = torch.empty((B, To, C0), dtype=torch.bfloat16, device=self.dev)
        arg = torch.empty((B, To, C0), dtype=torch.uint8, device=self.dev)
        gwx._check(lib.gwx_maxpool(gwx._ptr(a0), B, T1, C0, gwx._ptr(h), gwx._ptr(arg), st))
        tape["stem"] = (cols0, z0, ms0, a0, arg)
        tb = []
        for blk in self.blocks:
            s = blk["s"]
            z1, c1 = self._conv(h, blk["W116"], 5, s, 2)
            h1, ms1 = self._gn(z1, blk["g1"], blk["b1"], True)
            z2, c2 = self._conv(h1, blk["W216"], 5, 1, 2)
            if "Wd" in blk:
                zd, cd = self._conv(h, blk["Wd16"], 1, s, 0)
                sc, msd = self._gn(zd, blk["gd"], blk["bd"], False, out32=True)
                out, ms2 = self._gn(z2, blk["g2"], blk["b2"], True, res32=sc)
            else:
                zd = cd = msd = None
                out, ms2 = self._gn(z2, blk["g2"], blk["b2"], True, res16=h)
            tb.append((h, c1, z1, ms1, h1, c2, z2, ms2, cd, zd, msd, out))
            h = out
        tape["blocks"] = tb
        B, T, C = h.shape
        m = torch.empty((B, C), dtype=torch.bfloat16, device=self.dev)
        gwx._check(lib.gwx_mean_time(gwx._ptr(h), B, T, C, gwx._ptr(m), st))
        tape["m"] = m
        self.tape = tape
        return gwx.dense_bf16(m, self.W16["Wf"], self.P["bf"], act=gwx.ACT_NONE, out_dtype=out_dtype or torch.float32)

    def _scratch(self, nbytes):
        import torch
        buf = getattr(self, "_scratch_buf", None)
        if buf is None or buf.numel() < nbytes + 256:
            self._scratch_buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.dev)
        buf = self._scratch_buf
        off = (-buf.data_ptr()) % 256
        return buf[off:off + nbytes]

    def _gn_back(self, dy, z, ms, g):
        import torch
        gwx, lib = self.gwx, _lib.load()
        B, T, C = dy.shape
        dz = torch.empty_like(dy)
        dg, db = torch.empty(C, device=self.dev), torch.empty(C, device=self.dev)
        nb = lib.gwx_group_norm_backward_scratch(B, C, GROUPS)
        scratch = self._scratch(nb)
        gwx._check(lib.gwx_group_norm_backward(gwx._ptr(dy), gwx._ptr(z), B, T, C, GROUPS, gwx._ptr(ms), gwx._ptr(g),
                                               gwx._ptr(scratch), gwx._ptr(dz), gwx._ptr(dg), gwx._ptr(db),
                                               gwx._stream()))
        return dz, dg, db

    def _relu_mask(self, dy, out):
        import torch
        gwx = self.gwx
        d = torch.empty_like(dy)
        gwx._check(_lib.load().gwx_relu_mask(gwx._ptr(dy), gwx._ptr(out), dy.numel(), gwx._ptr(d), gwx._stream()))
        return d

    def _conv_back(self, dz, cols, W16, T, C, k, s, p, addend=None, x_in=None):
        """(dx [B][T][C] FP32, dW) of a convolution given dz [B][T_out][C_out]; x_in is the
        convolution's input when it ran as an implicit GEMM (cols None)."""
        import torch
        gwx = self.gwx
        if cols is None:
            B = x_in.shape[0]
            nb = _lib.load().gwx_conv1d_bf16_backward_workspace(B, T, C, W16.shape[0], k)
            return gwx.conv1d_bf16_backward(dz, x_in, W16, k, addend=addend,
                                            workspace=(self._scratch(nb), nb))
        B, To, Co = dz.shape
        dcols, dW, _ = gwx.dense_bf16_backward(cols, W16, None, dz.reshape(B * To, Co), act=gwx.ACT_NONE)
        dx = torch.empty((B, T, C), dtype=torch.float32, device=self.dev)
        gwx._check(_lib.load().gwx_col2im(gwx._ptr(dcols), B, T, C, k, s, p, W16.shape[1],
                                          gwx._ptr(addend) if addend is not None else None, gwx._ptr(dx),
                                          gwx._stream()))
        return dx, dW

    def backward(self, dc):
        """Gradients (dict name -> FP32 tensor, names of tensors()) for dL/dc = dc [B][out]."""
        import torch
        gwx, lib = self.gwx, _lib.load()
        st = gwx._stream()
        tape = self.tape
        G = {}
        m = tape["m"]
        dm, G["Wf"], G["bf"] = gwx.dense_bf16_backward(m, self.W16["Wf"], self.P["bf"], dc.contiguous(),
                                                       act=gwx.ACT_NONE)
        hT = tape["blocks"][-1][-1]
        B, T, C = hT.shape
        dh = torch.empty((B, T, C), dtype=torch.float32, device=self.dev)
        gwx._check(lib.gwx_mean_time_backward(gwx._ptr(dm), B, T, C, gwx._ptr(dh), st))
        for i in reversed(range(len(self.blocks))):
            blk = self.blocks[i]
            h, c1, z1, ms1, h1, c2, z2, ms2, cd, zd, msd, out = tape["blocks"][i]
            s = blk["s"]
            dsum = self._relu_mask(dh, out)
            dz2, G["%d.g2" % i], G["%d.b2" % i] = self._gn_back(dsum, z2, ms2, blk["g2"])
            dh1, G["%d.W2" % i] = self._conv_back(dz2, c2, blk["W216"], h1.shape[1], h1.shape[2], 5, 1, 2, x_in=h1)
            dh1 = self._relu_mask(dh1, h1)
            dz1, G["%d.g1" % i], G["%d.b1" % i] = self._gn_back(dh1, z1, ms1, blk["g1"])
            if "Wd" in blk:
                dzd, G["%d.gd" % i], G["%d.bd" % i] = self._gn_back(dsum, zd, msd, blk["gd"])
                dxs, G["%d.Wd" % i] = self._conv_back(dzd, cd, blk["Wd16"], h.shape[1], h.shape[2], 1, s, 0)
            else:
                dxs = dsum
            dh, G["%d.W1" % i] = self._conv_back(dz1, c1, blk["W116"], h.shape[1], h.shape[2], 5, s, 2, addend=dxs,
                                                 x_in=h)
        cols0, z0, ms0, a0, arg = tape["stem"]
        B, T1, C0 = a0.shape
        da0 = torch.empty((B, T1, C0), dtype=torch.float32, device=self.dev)
        gwx._check(lib.gwx_maxpool_backward(gwx._ptr(dh), gwx._ptr(arg), B, T1, C0, gwx._ptr(da0), st))
        da0 = self._relu_mask(da0, a0)
        dz0, G["g0"], G["b0"] = self._gn_back(da0, z0, ms0, self.P["g0"])
        _, G["W0"], _ = gwx.dense_bf16_backward(cols0, self.W16["W0"], None, dz0.reshape(B * T1, C0), want_dx=False,
                                                act=gwx.ACT_NONE)
        return G


__all__ = ["ResNet1D", "STAGES", "GROUPS"]
