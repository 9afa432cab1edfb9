"""Training driver of the transport surrogate (the BF16 forward/backward and
Adam kernels behind haar_mlp_train_step do the arithmetic; this only feeds
them mini-batches).

The surrogate maps a (vertex position, normal, view direction) to the
standardised coefficients of its transport at a fixed index set; the caller
provides the inputs raw [n, 9] and the standardised targets Y [n, 512] as
float32 device tensors."""
from __future__ import annotations


def fit(net, raw, Y, epochs: int, batch: int = 8192, lr=(1e-3, 3e-4, 1e-4), seed: int = 0, stream=None):
    """Adam on shuffled mini-batches for `epochs` passes over the n samples
    (the last partial batch of each epoch is dropped); the learning rate takes
    the values of `lr` in order, over equal parts of the run.
    Returns the mean training loss of the last epoch (a device scalar read
    once at the end)."""
    import torch
    n = raw.shape[0]
    steps_per_epoch = n // batch
    total = epochs * steps_per_epoch
    g = torch.Generator(device=raw.device).manual_seed(seed)
    rb = torch.empty((batch, raw.shape[1]), dtype=torch.float32, device=raw.device)
    yb = torch.empty((batch, Y.shape[1]), dtype=torch.float32, device=raw.device)
    loss_sum = torch.zeros(1, dtype=torch.float32, device=raw.device)
    loss = torch.zeros(1, dtype=torch.float32, device=raw.device)
    step = 0
    for e in range(epochs):
        perm = torch.randperm(n, generator=g, device=raw.device)
        if e == epochs - 1:
            loss_sum.zero_()
        for b in range(steps_per_epoch):
            sel = perm[b * batch:(b + 1) * batch]
            torch.index_select(raw, 0, sel, out=rb)
            torch.index_select(Y, 0, sel, out=yb)
            phase = min(len(lr) - 1, step * len(lr) // max(1, total))
            net.train_step(rb, yb, lr[phase], loss, stream)
            if e == epochs - 1:
                loss_sum += loss
            step += 1
    return float(loss_sum.item()) / max(1, steps_per_epoch)
