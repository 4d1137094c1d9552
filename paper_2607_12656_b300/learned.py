"""The learned part end to end: train the context model on a scene's own tokens with the
library's GPU training kernels, then freeze it to the integer model the bitstream carries
(Sec. 3.4.2; training loss = attribute rate of Eq. 9 in bits per token)."""
from __future__ import annotations

import numpy as np

from . import sgs
from .scenegen import kaiming_init


def train_and_freeze(ctx: sgs.Context, scene, depth: int, lanes: int, *, steps: int = 2000,
                     batch: int = 65536, seed: int = 1, lr: float = 1e-3, init_seed: int = 1,
                     return_losses: bool = False):
    import torch
    tokens = sgs.scene_tokens(scene.pos, scene.attr, depth)
    dev = torch.device("cuda", ctx.device)
    tok_dev = torch.from_numpy(tokens).to(dev)
    w = torch.from_numpy(sgs.pack_weights(kaiming_init(init_seed))).to(dev)
    adam = torch.zeros(2 * sgs.WEIGHTS_FLOATS, dtype=torch.float32, device=dev)
    losses = torch.zeros(max(steps, 1), dtype=torch.float32, device=dev)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    sgs.sgs_train(ctx, tok_dev, tokens.shape[0], lanes, w, adam, steps=steps, batch=batch, seed=seed,
                  lr=lr, loss_dev=losses)
    t1.record()
    weights = w.cpu().numpy()
    LAST_TRAIN.update(ms=t0.elapsed_time(t1), steps=steps, batch=batch,
                      final_bits=float(losses[max(steps, 1) - 1].item()))
    model = sgs.sgs_freeze(weights, tokens, lanes, seed)
    if return_losses:
        return model, weights, losses.cpu().numpy()[:steps]
    return model


def train_and_freeze_pe(ctx: sgs.Context, scene, depth: int, lanes: int, *, steps: int = 2000,
                        batch: int = 65536, seed: int = 1, lr: float = 1e-3, init_seed: int = 1,
                        return_losses: bool = False):
    """The position-aware model (Fourier positional embedding of the decoded voxel, Laplace
    head): train on the scene's own rows on the device, then freeze (SGS_MODEL_PE_BYTES)."""
    import torch
    from .scenegen import kaiming_init_pe
    tokens, coord = sgs.scene_rows(scene.pos, scene.attr, depth)
    dev = torch.device("cuda", ctx.device)
    tok_dev = torch.from_numpy(tokens).to(dev)
    crd_dev = torch.from_numpy(coord.view(np.int32)).to(dev)
    w = torch.from_numpy(sgs.pack_weights_pe(kaiming_init_pe(init_seed))).to(dev)
    adam = torch.zeros(2 * sgs.WEIGHTS_PE_FLOATS, dtype=torch.float32, device=dev)
    losses = torch.zeros(max(steps, 1), dtype=torch.float32, device=dev)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    sgs.sgs_train_pe(ctx, tok_dev, crd_dev, depth, tokens.shape[0], lanes, w, adam, steps=steps, batch=batch,
                     seed=seed, lr=lr, loss_dev=losses)
    t1.record()
    weights = w.cpu().numpy()
    LAST_TRAIN.update(ms=t0.elapsed_time(t1), steps=steps, batch=batch,
                      final_bits=float(losses[max(steps, 1) - 1].item()))
    model = sgs.sgs_freeze_pe(weights, tokens, coord, depth, lanes, seed)
    if return_losses:
        return model, weights, losses.cpu().numpy()[:steps]
    return model


# device time and final loss (bits per token) of the last train_and_freeze call
LAST_TRAIN = {}
