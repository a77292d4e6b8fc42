"""A small 3D convolutional network on the library's BF16 kernels (fwi_precond.h).

The learned gradient preconditioner maps the raw gradients and the current model,
(g_lambda, g_mu, lambda, mu) on the interior material grid, to a model update,
countering the lambda-mu cross-talk that the paper's biasing scheme (Sec. 3.3.3,
Eq. (25)) addresses by hand. ConvNet is that network: 3x3x3 convolutions with ReLU
between them, BF16 activations and weights, an FP32 master copy of the weights,
FP32 biases and gradients, trained with Adam on a mean squared error. Every
operation runs in the library's kernels; torch only holds the device memory and
gives the stream.
"""
from __future__ import annotations

import ctypes as C
import math

from .fwi import load_library


def _p(t):
    return C.c_void_p(t.data_ptr())


class ConvNet:
    """channels = (c_0, ..., c_L): L convolutions c_{l-1} -> c_l on a D x H x W grid, ReLU after
    all but the last. One sample per call ([C][D][H][W] tensors on `device`)."""

    def __init__(self, channels, shape, seed=0, device="cuda", lr=1e-3, betas=(0.9, 0.999), eps=1e-8):
        import torch

        if len(channels) < 2 or min(channels) < 1 or len(shape) != 3 or min(shape) < 1:
            raise ValueError("need at least two channel counts >= 1 and a 3D grid shape")
        self.lib = load_library()
        self.channels, self.shape = tuple(int(c) for c in channels), tuple(int(s) for s in shape)
        self.device = torch.device(device)
        self.lr, self.betas, self.eps, self.t = float(lr), betas, float(eps), 0
        gen = torch.Generator().manual_seed(seed)
        self.layers = []
        for cin, cout in zip(self.channels[:-1], self.channels[1:]):
            # He initialisation for ReLU networks: std = sqrt(2 / fan_in)
            master = (torch.randn(cout, cin, 27, generator=gen, dtype=torch.float32) *
                      math.sqrt(2.0 / (27 * cin))).to(self.device)
            layer = {"cin": cin, "cout": cout, "w32": master.contiguous(),
                     "w": torch.empty(cout, cin, 27, dtype=torch.bfloat16, device=self.device),
                     "b": torch.zeros(cout, dtype=torch.float32, device=self.device)}
            for k in ("w32", "b"):
                layer["m_" + k] = torch.zeros_like(layer[k])
                layer["v_" + k] = torch.zeros_like(layer[k])
                layer["g_" + k] = torch.zeros_like(layer[k])
            self._check(self.lib.fwi_nn_to_bf16(_p(layer["w32"]), layer["w32"].numel(), _p(layer["w"]),
                                                self._stream()))
            self.layers.append(layer)
        D, H, W = self.shape
        work = max(self.lib.fwi_nn_conv3d_backward_weight_work(l["cin"], l["cout"], D, H, W) for l in self.layers)
        self.work = torch.empty(int(work), dtype=torch.float32, device=self.device)
        self.red = torch.empty(1024, dtype=torch.float64, device=self.device)
        self.loss_dev = torch.zeros(1, dtype=torch.float64, device=self.device)

    def _stream(self):
        import torch

        return C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    @staticmethod
    def _check(status):
        if status != 0:
            raise RuntimeError(f"preconditioner kernel failed with status {status}")

    def to_bf16(self, x):
        """FP32 tensor -> BF16 tensor of the same shape, by the library's kernel."""
        import torch

        x = x.contiguous()
        y = torch.empty(x.shape, dtype=torch.bfloat16, device=self.device)
        self._check(self.lib.fwi_nn_to_bf16(_p(x), x.numel(), _p(y), self._stream()))
        return y

    def from_bf16(self, x):
        import torch

        y = torch.empty(x.shape, dtype=torch.float32, device=self.device)
        self._check(self.lib.fwi_nn_from_bf16(_p(x), x.numel(), _p(y), self._stream()))
        return y

    def forward(self, x):
        """Activations of every layer for the BF16 input x [c_0][D][H][W]; the last is the output."""
        import torch

        D, H, W = self.shape
        acts = [x.contiguous()]
        last = len(self.layers) - 1
        for i, l in enumerate(self.layers):
            y = torch.empty((l["cout"], D, H, W), dtype=torch.bfloat16, device=self.device)
            self._check(self.lib.fwi_nn_conv3d_forward(_p(acts[-1]), _p(l["w"]), _p(l["b"]), l["cin"], l["cout"], D, H,
                                                       W, int(i < last), _p(y), self._stream()))
            acts.append(y)
        return acts

    def __call__(self, x):
        """FP32 output for an FP32 or BF16 input."""
        import torch

        if x.dtype != torch.bfloat16:
            x = self.to_bf16(x)
        return self.from_bf16(self.forward(x)[-1])

    def train_step(self, x, target):
        """One Adam step on the loss sum (y - target)^2 / (2 n); returns the loss before the step.
        x: BF16 (or FP32) input, target: FP32 [c_L][D][H][W]."""
        import torch

        if x.dtype != torch.bfloat16:
            x = self.to_bf16(x)
        D, H, W = self.shape
        s = self._stream()
        acts = self.forward(x)
        target = target.contiguous()
        dy = torch.empty(target.shape, dtype=torch.float32, device=self.device)
        self._check(self.lib.fwi_nn_mse(_p(acts[-1]), _p(target), target.numel(), _p(dy), _p(self.loss_dev),
                                        _p(self.red), s))
        for i in range(len(self.layers) - 1, -1, -1):
            l = self.layers[i]
            if i < len(self.layers) - 1:  # through this layer's ReLU
                g = torch.empty_like(dy)
                self._check(self.lib.fwi_nn_relu_backward(_p(dy), _p(acts[i + 1]), dy.numel(), _p(g), s))
                dy = g
            self._check(self.lib.fwi_nn_conv3d_backward_weight(_p(dy), _p(acts[i]), l["cin"], l["cout"], D, H, W,
                                                               _p(l["g_w32"]), _p(l["g_b"]), _p(self.work), s))
            if i > 0:
                dx = torch.empty((l["cin"], D, H, W), dtype=torch.float32, device=self.device)
                self._check(self.lib.fwi_nn_conv3d_backward_data(_p(dy), _p(l["w"]), l["cin"], l["cout"], D, H, W,
                                                                 _p(dx), s))
                dy = dx
        self.t += 1
        b1, b2 = self.betas
        for l in self.layers:
            self._check(self.lib.fwi_nn_adam(_p(l["w32"]), _p(l["w"]), _p(l["g_w32"]), _p(l["m_w32"]), _p(l["v_w32"]),
                                             l["w32"].numel(), self.lr, b1, b2, self.eps, self.t, s))
            self._check(self.lib.fwi_nn_adam(_p(l["b"]), None, _p(l["g_b"]), _p(l["m_b"]), _p(l["v_b"]),
                                             l["b"].numel(), self.lr, b1, b2, self.eps, self.t, s))
        return float(self.loss_dev.item())


class _Conv:
    """One 3x3x3 convolution layer: BF16 weights with an FP32 master copy, FP32 bias, and
    their gradients and Adam moments."""

    def __init__(self, lib, cin, cout, relu, gen, device):
        import torch

        self.cin, self.cout, self.relu = int(cin), int(cout), bool(relu)
        # He initialisation for ReLU networks: std = sqrt(2 / fan_in)
        self.w32 = (torch.randn(cout, cin, 27, generator=gen, dtype=torch.float32) *
                    math.sqrt(2.0 / (27 * cin))).to(device).contiguous()
        self.w = torch.empty(cout, cin, 27, dtype=torch.bfloat16, device=device)
        self.b = torch.zeros(cout, dtype=torch.float32, device=device)
        for k in ("w32", "b"):
            setattr(self, "g_" + k, torch.zeros_like(getattr(self, k)))
            setattr(self, "m_" + k, torch.zeros_like(getattr(self, k)))
            setattr(self, "v_" + k, torch.zeros_like(getattr(self, k)))
        self.lib = lib

    def params(self):
        return self.w32.numel() + self.b.numel()


class UNet:
    """A three-level 3D U-Net on the library's BF16 kernels: at each level two 3x3x3
    convolutions with ReLU, 2x average pooling down, nearest-neighbour upsampling up, and
    skip connections that concatenate the upsampled field with the same level's encoder
    output along the channels; the last convolution is linear. widths = (w0, w1, w2) are
    the channels at full, half and quarter resolution. One sample per call
    ([C][D][H][W] tensors on `device`); training uses sum (y - t)^2 / (2 n) and Adam."""

    def __init__(self, cin, cout, widths, shape, seed=0, device="cuda", lr=1e-3, betas=(0.9, 0.999), eps=1e-8):
        import torch

        if len(widths) != 3 or min(widths) < 1 or cin < 1 or cout < 1 or len(shape) != 3 or min(shape) < 1:
            raise ValueError("need three widths >= 1, cin, cout >= 1 and a 3D grid shape")
        self.lib = load_library()
        self.device = torch.device(device)
        self.cin, self.cout = int(cin), int(cout)
        w0, w1, w2 = (int(w) for w in widths)
        self.widths = (w0, w1, w2)
        s0 = tuple(int(s) for s in shape)
        s1 = tuple((s + 1) // 2 for s in s0)
        s2 = tuple((s + 1) // 2 for s in s1)
        self.shapes = (s0, s1, s2)
        self.lr, self.betas, self.eps, self.t = float(lr), betas, float(eps), 0
        gen = torch.Generator().manual_seed(seed)
        mk = lambda a, b, r: _Conv(self.lib, a, b, r, gen, self.device)  # noqa: E731
        # (name, layer, level)
        self.convs = [("e0a", mk(cin, w0, True), 0), ("e0b", mk(w0, w0, True), 0),
                      ("e1a", mk(w0, w1, True), 1), ("e1b", mk(w1, w1, True), 1),
                      ("ba", mk(w1, w2, True), 2), ("bb", mk(w2, w2, True), 2),
                      ("d1a", mk(w2 + w1, w1, True), 1), ("d1b", mk(w1, w1, True), 1),
                      ("d0a", mk(w1 + w0, w0, True), 0), ("d0b", mk(w0, cout, False), 0)]
        self.layer = {n: l for n, l, _ in self.convs}
        self.level = {n: lv for n, _, lv in self.convs}
        for _, l, _ in self.convs:
            self._check(self.lib.fwi_nn_to_bf16(_p(l.w32), l.w32.numel(), _p(l.w), self._stream()))
        work = max(self.lib.fwi_nn_conv3d_backward_weight_work(l.cin, l.cout, *self.shapes[lv])
                   for _, l, lv in self.convs)
        self.work = torch.empty(int(work), dtype=torch.float32, device=self.device)
        self.red = torch.empty(1024, dtype=torch.float64, device=self.device)
        self.loss_dev = torch.zeros(1, dtype=torch.float64, device=self.device)

    def num_params(self):
        return sum(l.params() for _, l, _ in self.convs)

    def _stream(self):
        import torch

        return C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    _check = staticmethod(ConvNet._check)
    to_bf16 = ConvNet.to_bf16
    from_bf16 = ConvNet.from_bf16

    def _conv(self, name, x, out):
        l, lv = self.layer[name], self.level[name]
        self._check(self.lib.fwi_nn_conv3d_forward(_p(x), _p(l.w), _p(l.b), l.cin, l.cout, *self.shapes[lv],
                                                   int(l.relu), _p(out), self._stream()))
        return out

    def forward(self, x):
        """BF16 activations of every layer for the BF16 input x [cin][D][H][W], by name; 'y'
        is the output. cat0 / cat1 hold [upsampled deeper field, encoder output] of levels 0 / 1."""
        import torch

        (s0, s1, s2), (w0, w1, w2) = self.shapes, self.widths
        bf = lambda c, s: torch.empty((c, *s), dtype=torch.bfloat16, device=self.device)  # noqa: E731
        st = self._stream()
        a = {"x": x.contiguous()}
        a["e0a"] = self._conv("e0a", a["x"], bf(w0, s0))
        a["cat0"] = bf(w1 + w0, s0)
        self._conv("e0b", a["e0a"], a["cat0"][w1:])
        a["p0"] = bf(w0, s1)
        self._check(self.lib.fwi_nn_pool2_forward(_p(a["cat0"][w1:]), w0, *s0, _p(a["p0"]), st))
        a["e1a"] = self._conv("e1a", a["p0"], bf(w1, s1))
        a["cat1"] = bf(w2 + w1, s1)
        self._conv("e1b", a["e1a"], a["cat1"][w2:])
        a["p1"] = bf(w1, s2)
        self._check(self.lib.fwi_nn_pool2_forward(_p(a["cat1"][w2:]), w1, *s1, _p(a["p1"]), st))
        a["ba"] = self._conv("ba", a["p1"], bf(w2, s2))
        a["bb"] = self._conv("bb", a["ba"], bf(w2, s2))
        self._check(self.lib.fwi_nn_upsample2_forward(_p(a["bb"]), w2, *s1, _p(a["cat1"][:w2]), st))
        a["d1a"] = self._conv("d1a", a["cat1"], bf(w1, s1))
        a["d1b"] = self._conv("d1b", a["d1a"], bf(w1, s1))
        self._check(self.lib.fwi_nn_upsample2_forward(_p(a["d1b"]), w1, *s0, _p(a["cat0"][:w1]), st))
        a["d0a"] = self._conv("d0a", a["cat0"], bf(w0, s0))
        a["y"] = self._conv("d0b", a["d0a"], bf(self.cout, s0))
        return a

    def __call__(self, x):
        """FP32 output for an FP32 or BF16 input."""
        import torch

        if x.dtype != torch.bfloat16:
            x = self.to_bf16(x)
        return self.from_bf16(self.forward(x)["y"])

    def _backward(self, name, dy, x, need_dx):
        """weight and bias gradients of layer `name` from dy (FP32, pre-activation) and its
        input x; returns the FP32 gradient with respect to x when asked."""
        import torch

        l, lv = self.layer[name], self.level[name]
        s = self._stream()
        self._check(self.lib.fwi_nn_conv3d_backward_weight(_p(dy), _p(x), l.cin, l.cout, *self.shapes[lv],
                                                           _p(l.g_w32), _p(l.g_b), _p(self.work), s))
        if not need_dx:
            return None
        dx = torch.empty((l.cin, *self.shapes[lv]), dtype=torch.float32, device=self.device)
        self._check(self.lib.fwi_nn_conv3d_backward_data(_p(dy), _p(l.w), l.cin, l.cout, *self.shapes[lv], _p(dx), s))
        return dx

    def _relu_back(self, g, y):
        import torch

        out = torch.empty_like(g)
        self._check(self.lib.fwi_nn_relu_backward(_p(g), _p(y), g.numel(), _p(out), self._stream()))
        return out

    def backward(self, a, dy):
        """Gradients of every layer's weights and bias for output gradient dy (FP32), from
        the activations a of forward()."""
        import torch

        (s0, s1, s2), (w0, w1, w2) = self.shapes, self.widths
        st = self._stream()
        g = self._backward("d0b", dy, a["d0a"], True)
        g = self._relu_back(g, a["d0a"])
        gcat0 = self._backward("d0a", g, a["cat0"], True)       # [w1 + w0][s0]
        g = torch.empty((w1, *s1), dtype=torch.float32, device=self.device)
        self._check(self.lib.fwi_nn_upsample2_backward(_p(gcat0[:w1]), w1, *s0, 0, _p(g), st))
        g = self._relu_back(g, a["d1b"])
        g = self._backward("d1b", g, a["d1a"], True)
        g = self._relu_back(g, a["d1a"])
        gcat1 = self._backward("d1a", g, a["cat1"], True)       # [w2 + w1][s1]
        g = torch.empty((w2, *s2), dtype=torch.float32, device=self.device)
        self._check(self.lib.fwi_nn_upsample2_backward(_p(gcat1[:w2]), w2, *s1, 0, _p(g), st))
        g = self._relu_back(g, a["bb"])
        g = self._backward("bb", g, a["ba"], True)
        g = self._relu_back(g, a["ba"])
        g = self._backward("ba", g, a["p1"], True)               # [w1][s2]
        # the level-1 encoder output feeds the pooling and the skip: its gradients add
        ge1 = gcat1[w2:].contiguous()
        self._check(self.lib.fwi_nn_pool2_backward(_p(g), w1, *s1, 1, _p(ge1), st))
        g = self._relu_back(ge1, a["cat1"][w2:])
        g = self._backward("e1b", g, a["e1a"], True)
        g = self._relu_back(g, a["e1a"])
        g = self._backward("e1a", g, a["p0"], True)              # [w0][s1]
        ge0 = gcat0[w1:].contiguous()
        self._check(self.lib.fwi_nn_pool2_backward(_p(g), w0, *s0, 1, _p(ge0), st))
        g = self._relu_back(ge0, a["cat0"][w1:])
        g = self._backward("e0b", g, a["e0a"], True)
        g = self._relu_back(g, a["e0a"])
        self._backward("e0a", g, a["x"], False)

    def train_step(self, x, target):
        """One Adam step on sum (y - target)^2 / (2 n); returns the loss before the step."""
        import torch

        if x.dtype != torch.bfloat16:
            x = self.to_bf16(x)
        s = self._stream()
        a = self.forward(x)
        target = target.contiguous()
        dy = torch.empty(target.shape, dtype=torch.float32, device=self.device)
        self._check(self.lib.fwi_nn_mse(_p(a["y"]), _p(target), target.numel(), _p(dy), _p(self.loss_dev),
                                        _p(self.red), s))
        self.backward(a, dy)
        self.t += 1
        b1, b2 = self.betas
        for _, l, _ in self.convs:
            self._check(self.lib.fwi_nn_adam(_p(l.w32), _p(l.w), _p(l.g_w32), _p(l.m_w32), _p(l.v_w32), l.w32.numel(),
                                             self.lr, b1, b2, self.eps, self.t, s))
            self._check(self.lib.fwi_nn_adam(_p(l.b), None, _p(l.g_b), _p(l.m_b), _p(l.v_b), l.b.numel(), self.lr,
                                             b1, b2, self.eps, self.t, s))
        return float(self.loss_dev.item())


def precond_inputs(g_lambda, g_mu, lam, mu, lam_bg, mu_bg):
    """The network input [4][D][H][W] (FP32, on the gradients' device) for one model: the
    misfit gradients scaled together by their largest magnitude (their ratio, where the
    lambda-mu cross-talk shows, is kept), and the model as relative perturbations of the
    background values lam_bg, mu_bg."""
    import torch

    gl = torch.as_tensor(g_lambda).to(torch.float64)
    gm = torch.as_tensor(g_mu).to(gl.device, torch.float64)
    scale = torch.maximum(gl.abs().max(), gm.abs().max()).clamp_min(1e-300)
    lam = torch.as_tensor(lam).to(gl.device, torch.float64)
    mu = torch.as_tensor(mu).to(gl.device, torch.float64)
    x = torch.stack([gl / scale, gm / scale, lam / lam_bg - 1.0, mu / mu_bg - 1.0])
    return x.to(torch.float32).contiguous()


def precond_targets(lam_true, mu_true, lam, mu, lam_bg, mu_bg):
    """The training target [2][D][H][W]: the remaining model error (true minus current) of
    lambda and mu, relative to the background values."""
    import torch

    lt = torch.as_tensor(lam_true).to(torch.float64)
    d = lt.device
    t = torch.stack([(lt - torch.as_tensor(lam).to(d, torch.float64)) / lam_bg,
                     (torch.as_tensor(mu_true).to(d, torch.float64) - torch.as_tensor(mu).to(d, torch.float64)) / mu_bg])
    return t.to(torch.float32).contiguous()


def learned_update(net, g_lambda, g_mu, lam, mu, lam_bg, mu_bg):
    """The model update (d_lambda, d_mu) in Pa that the network proposes for a model and its
    misfit gradients (FP64 tensors on the network's device)."""
    import torch

    y = net(precond_inputs(g_lambda, g_mu, lam, mu, lam_bg, mu_bg).to(net.device)).to(torch.float64)
    return y[0] * lam_bg, y[1] * mu_bg
