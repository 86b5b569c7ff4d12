"""3D U-Net that maps the normalised backprojection A^T b / (A^T A 1) to a CGLS warm start.

Four levels with 16, 32, 64, 128 channels; two 3x3x3 convolutions (+ bias, ReLU) per level;
2x2x2 max pooling down, nearest-neighbour x2 upsampling followed by a 3x3x3 convolution that
halves the channels up, concatenation with the skip connection, two convolutions; a final
3x3x3 convolution whose channel 0 is added to the input (the network learns a correction of
the normalised backprojection). Inside the network the input and the correction are
multiplied by a fixed scale (set from the training targets) so that activations are O(1). Activations are channels-last bf16 [n, d, h, w, c]; every
convolution (forward and both gradients) runs in the tensor-core kernels of libkct_conv;
pooling, upsampling, concatenation and the loss are torch glue.

The single input channel is padded with zeros to 16 channels (the convolution kernels take
multiples of 16); the final convolution has 16 output channels of which channel 0 is used.
"""
from __future__ import annotations

import math

import torch

from . import conv


def _conv_param(cout, cin, gen):
    std = math.sqrt(2.0 / (27 * cin))                   # He initialisation for ReLU layers
    w = torch.randn((cout, 27, cin), generator=gen) * std
    return torch.nn.Parameter(w), torch.nn.Parameter(torch.zeros(cout))


class UNet3D(torch.nn.Module):
    def __init__(self, base: int = 16, levels: int = 4, seed: int = 0):
        super().__init__()
        gen = torch.Generator().manual_seed(seed)
        self.levels = levels
        ch = [base * 2 ** i for i in range(levels)]
        self.ch = ch
        self.names = []

        def add(name, cout, cin):
            w, b = _conv_param(cout, cin, gen)
            self.register_parameter(name + "_w", w)
            self.register_parameter(name + "_b", b)
            self.names.append(name)

        cin = base                                       # padded input channels
        for i in range(levels):
            add(f"enc{i}a", ch[i], cin)
            add(f"enc{i}b", ch[i], ch[i])
            cin = ch[i]
        for i in range(levels - 2, -1, -1):
            add(f"up{i}", ch[i], ch[i + 1])
            add(f"dec{i}a", ch[i], 2 * ch[i])
            add(f"dec{i}b", ch[i], ch[i])
        add("head", base, base)
        with torch.no_grad():                            # start as the identity correction
            self.head_w.zero_()
        # inputs and corrections are scaled by this factor inside the network, so that its
        # activations are O(1) whatever the attenuation scale of the data
        self.register_buffer("scale", torch.ones(()))

    def _c(self, name, x, relu=True):
        return conv.conv3d(x, getattr(self, name + "_w"), getattr(self, name + "_b"), relu)

    @staticmethod
    def _pool(x):
        n, d, h, w, c = x.shape
        return x.view(n, d // 2, 2, h // 2, 2, w // 2, 2, c).amax(dim=(2, 4, 6))

    @staticmethod
    def _up(x):
        return x.repeat_interleave(2, dim=1).repeat_interleave(2, dim=2).repeat_interleave(2, dim=3).contiguous()

    def forward(self, inp: torch.Tensor) -> torch.Tensor:
        """inp: float [n, d, h, w] (normalised backprojection) -> float [n, d, h, w]."""
        n, d, h, w = inp.shape
        x = torch.zeros((n, d, h, w, self.ch[0]), dtype=torch.bfloat16, device=inp.device)
        x[..., 0] = (inp * self.scale).to(torch.bfloat16)
        skips = []
        for i in range(self.levels):
            if i > 0:
                x = self._pool(x)
            x = self._c(f"enc{i}a", x)
            x = self._c(f"enc{i}b", x)
            skips.append(x)
        for i in range(self.levels - 2, -1, -1):
            x = self._c(f"up{i}", self._up(x))
            x = torch.cat([x, skips[i]], dim=-1).contiguous()
            x = self._c(f"dec{i}a", x)
            x = self._c(f"dec{i}b", x)
        y = self._c("head", x, relu=False)
        return inp + y[..., 0].float() / self.scale
