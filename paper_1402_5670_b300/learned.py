"""Training loop of the learned shrinkage (host orchestration of the sl_mlp_* calls).

Noisy/clean pairs come from the transform itself: a seeded synthetic clean signal and
its noisy copy are both transformed on the GPU, and the MLP learns to map the noisy
coefficients to the clean ones. Sample indices are drawn by a seeded torch generator
on the device and passed to the library.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

from . import synth
from .shearlet import MLP, Bank


def make_pairs(bank: Bank, sigmas: Sequence[float], seeds: Sequence[int]):
    """[(noisy_coeffs, clean_coeffs, sigma)] on the device, one pair per (seed, sigma)."""
    import torch
    pairs = []
    for sd in seeds:
        clean = (synth.piecewise_smooth_image(bank.dims, sd) if bank.ndim == 2
                 else synth.moving_ellipses_volume(bank.dims, sd))
        cg = torch.from_numpy(clean).cuda()
        Cc = bank.forward(cg)
        for i, sg in enumerate(sigmas):
            noisy = synth.add_noise(clean, sg, 7919 * sd + i)
            Cn = bank.forward(torch.from_numpy(noisy).cuda())
            pairs.append((Cn, Cc, float(sg)))
    return pairs


def train(mlp: MLP, pairs, steps: int, batch: int = 16384, lr: float = 2e-3,
          seed: int = 0, lr_final: float = 2e-4) -> List[float]:
    """Adam on random coefficient samples (subbands j >= 1) cycling over the pairs;
    the learning rate decays geometrically from lr to lr_final. Returns the losses."""
    import torch
    bank = mlp.bank
    gen = torch.Generator(device="cuda")
    gen.manual_seed(int(seed))
    span = (bank.R - 1) * bank.N
    loss = torch.zeros(1, device="cuda")
    hist = []
    for k in range(steps):
        Cn, Cc, sg = pairs[k % len(pairs)]
        idx = (torch.randint(0, span, (batch,), generator=gen, device="cuda")
               + bank.N).to(torch.int32)
        rate = lr * (lr_final / lr) ** (k / max(1, steps - 1))
        mlp.train_step(Cn, Cc, sg, idx, rate, loss_out=loss)
        if k % 50 == 0 or k == steps - 1:
            hist.append(float(loss.item()))
    return hist
