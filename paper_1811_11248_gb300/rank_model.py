"""Learned rank predictor: data collection, GPU training and inference.

The factorization records, for every cluster it eliminates, 8 features of
the scaled block row and the rank its column-pivoted QR found
(``hs_options.record_ranks`` / ``Handle.rank_samples``).  A three-layer
perceptron of width 64 is fitted to the fraction rank / s with the library's
own CUDA kernels (``hs_mlp_train``: minibatch forward + backpropagation +
Adam) and evaluated with ``hs_mlp_forward``.  Inputs are standardised with
the training set's mean and deviation, which the model keeps.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import hsolve, inputs


@dataclass
class RankModel:
    mu: np.ndarray      # float32[8] feature means of the training set
    sd: np.ndarray      # float32[8] feature deviations (>= 1e-6)
    params: np.ndarray  # float32[4801] network parameters

    def normalise(self, feat):
        return ((np.asarray(feat, np.float32) - self.mu) / self.sd).astype(np.float32)

    def predict_fraction(self, feat):
        """Network output for raw features (GPU forward kernel)."""
        import torch
        x = torch.from_numpy(self.normalise(feat)).cuda()
        th = torch.from_numpy(np.ascontiguousarray(self.params, np.float32)).cuda()
        y = torch.empty(len(x), dtype=torch.float32, device="cuda")
        hsolve.hs_mlp_forward(th, x, len(x), y, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        return y.cpu().numpy()

    def predict_rank(self, feat, size):
        """Rank estimate: round(fraction * s), clipped to [0, min(s, fill columns)]."""
        feat = np.asarray(feat, np.float32)
        f = self.predict_fraction(feat)
        cap = np.minimum(np.asarray(size), feat[:, 2]).astype(np.int64)
        return np.clip(np.rint(f * np.asarray(size)), 0, cap).astype(np.int32)

    def save(self, path):
        np.savez(path, mu=self.mu, sd=self.sd, params=self.params)

    @staticmethod
    def load(path):
        z = np.load(path)
        return RankModel(z["mu"], z["sd"], z["params"])

    def packed(self):
        """mu (8), sd (8), params (4801) as one float32 vector."""
        return np.concatenate([self.mu, self.sd, self.params]).astype(np.float32)


def collect(problem, tol=1e-2, depth=-1, precision=hsolve.HS_PREC_FP64, stream=None):
    """Set up `problem` with rank recording; -> (features, ranks, sizes)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    opt = hsolve.hs_default_options(tol=tol, depth=depth, mem=hsolve.HS_MEM_HOST, coords=problem.coords,
                                    stream=st, precision=precision, record_ranks=1)
    h = hsolve.hs_setup(problem.n, problem.rowptr, problem.col, problem.val, opt=opt)
    try:
        return h.rank_samples()
    finally:
        h.close()


def collect_batched(problems, tol=1e-2, precision=hsolve.HS_PREC_FP64, stream=None):
    """Rank samples of several independent problems set up as one batch."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    pp, A = inputs.block_diagonal(problems)
    opt = hsolve.hs_default_options(tol=tol, mem=hsolve.HS_MEM_HOST, coords=A.coords, stream=st,
                                    precision=precision, record_ranks=1)
    h = hsolve.hs_setup_batched(pp, A.n, A.rowptr, A.col, A.val, opt=opt)
    try:
        return h.rank_samples()
    finally:
        h.close()


def fit(feat, rank, size, epochs=30, batch=256, lr=2e-3, seed=0):
    """Train on recorded samples with the GPU kernels -> (RankModel, losses)."""
    feat = np.asarray(feat, np.float32)
    mu = feat.mean(axis=0).astype(np.float32)
    sd = np.maximum(feat.std(axis=0), 1e-6).astype(np.float32)
    model = RankModel(mu, sd, inputs.mlp_init_params(seed).astype(np.float32))
    x = model.normalise(feat)
    t = (np.asarray(rank, np.float32) / np.maximum(np.asarray(size, np.float32), 1.0)).astype(np.float32)
    b = min(batch, len(t))
    order = inputs.mlp_batch_order(len(t), b, epochs, seed + 1)
    model.params, losses = hsolve.hs_mlp_train(model.params, x, t, order, b, lr)
    return model, losses


def accuracy(model, feat, rank, size):
    """Exact-match share, mean absolute error (ranks) and the mean absolute
    error of the best constant fraction (the baseline without the network)."""
    pred = model.predict_rank(feat, size)
    rank = np.asarray(rank)
    frac = np.asarray(rank, np.float64) / np.maximum(np.asarray(size), 1)
    const = np.clip(np.rint(np.median(frac) * np.asarray(size)), 0, None)
    return {"exact": float(np.mean(pred == rank)), "mae": float(np.mean(np.abs(pred - rank))),
            "mae_constant": float(np.mean(np.abs(const - rank))), "n": int(len(rank))}
