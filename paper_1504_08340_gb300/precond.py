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
