"""Training driver for the learned candidate proposal (argument marshalling only).

Every computation runs in the library: signals are synthesised on the device from seeded
supports, coefficients and noise (``omp_synthesize_signals``), labelled by plain OMP
(``omp_solve_batch_trace``, which also records each step's normalised residual drop), the drop
thresholds tau_k are the given quantile of those drops per step (``omp_proposal_calibrate``), and
the network is trained with the library's forward/backward kernels and AdamW
(``omp_proposal_train_step``). The host only draws the seeded random inputs.
"""
from __future__ import annotations

import concurrent.futures
import dataclasses
import time

import numpy as np

from . import omp


@dataclasses.dataclass
class TrainReport:
    n_signals: int
    epochs: int
    steps: int
    losses: list          # mean loss of each epoch
    tau: np.ndarray       # calibrated thresholds
    seconds_data: float
    seconds_train: float


def init_weights(N: int, hidden: int, S: int, seed: int = 0, M: int = None):
    """Seeded initial parameters: uniform(+-1/sqrt(fan_in)) weights scaled down by 1/8 so the
    network starts as a small correction, zero hidden bias, an output bias at the prior logit
    log(S / (N - S)) of an atom being in the support, and a skip scale beta that makes |x| (whose
    typical size is 1/sqrt(M) for unit vectors) span a few logits, so the initial proposal is the
    top-K of |A^T y|."""
    rng = np.random.default_rng(np.random.SeedSequence(seed, spawn_key=(9,)))
    W1 = rng.uniform(-1, 1, size=(hidden, N)).astype(np.float32) / np.float32(8 * np.sqrt(N))
    W2 = rng.uniform(-1, 1, size=(N, hidden)).astype(np.float32) / np.float32(8 * np.sqrt(hidden))
    b1 = np.zeros(hidden, dtype=np.float32)
    b2 = np.full(N, np.log(S / max(N - S, 1)), dtype=np.float32)
    beta = np.array([4.0 * np.sqrt(M if M else N)], dtype=np.float32)
    return W1, b1, W2, b2, beta


def _to_dev(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().to(dev, non_blocking=True)


def make_training_set(solver_h, A_dev, w, n_signals: int, chunk: int, seed: int = 0,
                      threads: int = 8):
    """Synthesise n_signals training signals on the device and label them with plain OMP.

    The labels are the supports of the dense solve (Alg. 1, no proposal) of the handle given. On
    a BF16 or FP8 handle the FP32 rescoring makes every pick the FP32 path's (the GPU tests assert
    bit-identical supports), so the labels are those of plain FP32 OMP at the quantised form's
    cost.

    Returns (Y (n x M), labels (n x S int32), drops (n x S float32)) as device tensors."""
    import torch
    from workloads import gen
    dev = A_dev.device
    n_chunks = (n_signals + chunk - 1) // chunk
    Y = torch.empty((n_signals, w.M), dtype=torch.float32, device=dev)
    labels = torch.empty((n_signals, w.S), dtype=torch.int32, device=dev)
    drops = torch.empty((n_signals, w.S), dtype=torch.float32, device=dev)
    X = torch.empty((chunk, w.S), dtype=torch.float32, device=dev)

    def draw(c):
        n = min(chunk, n_signals - c * chunk)
        return c, n, gen.training_batch(w, n, chunk_id=c, seed=seed)

    with concurrent.futures.ThreadPoolExecutor(max_workers=threads) as ex:
        for c, n, (sup, coef, noise) in ex.map(draw, range(n_chunks)):
            lo = c * chunk
            sup_d, coef_d, noise_d = _to_dev(sup, dev), _to_dev(coef, dev), _to_dev(noise, dev)
            omp.omp_synthesize_signals(A_dev, sup_d, coef_d, noise_d, Y[lo:lo + n])
            omp.omp_solve_batch_trace(solver_h, A_dev, Y[lo:lo + n], w.S, w.eps, X[:n],
                                      labels[lo:lo + n], drops[lo:lo + n])
    torch.cuda.synchronize(dev)
    return Y, labels, drops


def train(solver_h, proposal: "omp.Proposal", A_dev, w, n_signals: int = 1 << 20,
          epochs: int = 3, batch: int = 4096, chunk: int = 16384, quantile: float = 1e-3,
          seed: int = 0, log=None) -> TrainReport:
    """Label n_signals generated signals with plain OMP, calibrate tau, and train for `epochs`
    passes of minibatches of `batch` signals (seeded block order per epoch)."""
    import torch
    dev = A_dev.device
    t0 = time.perf_counter()
    Y, labels, drops = make_training_set(solver_h, A_dev, w, n_signals, chunk, seed)
    proposal.calibrate(drops, quantile)
    tau = proposal.get_thresholds(w.S)
    t1 = time.perf_counter()
    rng = np.random.default_rng(np.random.SeedSequence(seed, spawn_key=(10,)))
    nblk = n_signals // batch
    step_loss = torch.zeros((epochs, max(nblk, 1)), dtype=torch.float32, device=dev)
    losses = []
    steps = 0
    for e in range(epochs):
        for i, blk in enumerate(rng.permutation(nblk)):
            lo = int(blk) * batch
            proposal.train_step(A_dev, Y[lo:lo + batch], labels[lo:lo + batch], step_loss[e, i:i + 1])
            steps += 1
        losses.append(float(step_loss[e].cpu().numpy()[:nblk].mean()) if nblk else float("nan"))
        if log:
            log(f"epoch {e}: mean loss {losses[-1]:.6g}")
    torch.cuda.synchronize(dev)
    t2 = time.perf_counter()
    return TrainReport(n_signals, epochs, steps, losses, tau, t1 - t0, t2 - t1)
