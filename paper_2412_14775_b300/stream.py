"""Convenience wrapper: one RFI flagging context plus torch-allocated outputs.

Device memory comes from torch; all computation is the library's CUDA kernels,
reached through the C ABI (binding.py)."""
from . import binding as B

_TORCH_DTYPE = {B.RFI_C64: "float32", B.RFI_C32H: "float16"}


class RfiStream:
    """One stream of `stations` x `channels` rows, window M, averaging factor K."""

    def __init__(self, stations, channels, M, K, thresholds, dtype="f32", **options):
        self.stations, self.channels, self.M, self.K = stations, channels, M, K
        self.dtype = B._dtype(dtype)
        self.ctx = B.rfi_create_ex(stations, channels, M, K, thresholds, self.dtype, **options)
        self.R = B.rfi_rows(self.ctx)
        self.options = B.rfi_get_options(self.ctx)
        self.F = self.options["window_F"]
        # flag bits a completed window adds to a call's output: M, or the hop H when
        # windows overlap (the samples that became final)
        self.bits_per_window = self.options["window_hop"] or M

    # -- outputs ------------------------------------------------------------------
    def outputs_for(self, T):
        return B.rfi_outputs_for(self.ctx, T)

    def windows_for(self, T):
        """(n_win, first_sample) of the next block of T samples."""
        return B.rfi_windows_for(self.ctx, T)

    def alloc_outputs(self, T, device="cuda", pin_memory=False):
        """Outputs of the NEXT block of T samples (their sizes depend on the stream's
        position when windows or bins straddle blocks)."""
        import torch
        n_out = self.outputs_for(T)
        n_win = self.windows_for(T)[0]
        kw = dict(device=device) if device != "cpu" else dict(pin_memory=pin_memory)
        return dict(
            flags=torch.empty((self.R, (n_win * self.bits_per_window + 31) // 32),
                              dtype=torch.int32, **kw),
            avg=torch.empty((self.R, n_out, 4, 2), dtype=torch.float32, **kw),
            weight=torch.empty((self.R, n_out), dtype=torch.float32, **kw),
            stats=torch.empty((3, self.R // self.F, n_win), dtype=torch.float32, **kw))

    def _T(self, vis):
        if vis.shape[-2:] != (4, 2):
            raise ValueError("visibilities must end in [4, 2] (correlation, re/im)")
        return vis.shape[-3]

    # -- processing ---------------------------------------------------------------
    def process(self, vis, out=None, stream=None):
        """vis: CUDA tensor [..., T, 4, 2] with R rows in front, in the context dtype."""
        T = self._T(vis)
        if out is None:
            out = self.alloc_outputs(T, device=vis.device)
        n_out = out["weight"].shape[1]
        B.rfi_process_block(self.ctx, vis, T, out["flags"], out["avg"] if n_out else None,
                            out["weight"] if n_out else None, out["stats"], stream)
        return out

    def process_host(self, vis, out=None, stream=None):
        """vis: host tensor (pinned for overlap); outputs are host tensors."""
        T = self._T(vis)
        if out is None:
            out = self.alloc_outputs(T, device="cpu", pin_memory=vis.is_pinned())
        n_out = out["weight"].shape[1]
        B.rfi_process_block_host(self.ctx, vis, T, out["flags"], out["avg"] if n_out else None,
                                 out["weight"] if n_out else None, out["stats"], stream)
        return out

    def set_adaptation(self, alpha=1.0 / 64, k_sigma=3.0, n_warm=32):
        """Parameters of the online SK thresholds (contexts created with adaptive=1)."""
        B.rfi_set_adaptation(self.ctx, alpha, k_sigma, n_warm)

    def adaptive_state(self, state=None):
        """Read, or with `state` write, the per-row (n, mean tau, mean tau^2, 0)."""
        return B.rfi_adaptive_state(self.ctx, state)

    def reset(self):
        B.rfi_reset(self.ctx)

    def close(self):
        if self.ctx:
            B.rfi_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
