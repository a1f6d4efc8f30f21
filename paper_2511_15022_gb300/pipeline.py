"""Double-buffered host-to-device input stream for training loops.

While step k runs on the compute stream, the copy of step k + 1's input (from pinned host
memory) runs on a separate copy stream; CUDA events order each buffer's copy before its
use and each reuse of a buffer after the step that read it.  Only device memory, streams
and events are involved; the optimisation step itself runs in the library's kernels.
"""
from __future__ import annotations

from typing import Optional

import torch


class InputPipeline:
    """`depth` device buffers of one shape, filled in turn on a copy stream."""

    def __init__(self, shape, dtype, device, depth: int = 2):
        self.device = torch.device(device)
        self.bufs = [torch.empty(shape, dtype=dtype, device=self.device) for _ in range(depth)]
        self.copy_stream = torch.cuda.Stream(device=self.device)
        self.ready = [torch.cuda.Event() for _ in range(depth)]   # copy into buffer i done
        self.free = [torch.cuda.Event() for _ in range(depth)]    # last reader of i done
        self.used = [False] * depth
        self.head = 0   # next buffer to fill
        self.tail = 0   # next buffer to hand out
        self.pending = 0

    def put(self, host: torch.Tensor, stream: Optional[torch.cuda.Stream] = None):
        """Start copying `host` (pinned for the copy to be asynchronous) into the next
        buffer."""
        if self.pending == len(self.bufs):
            raise RuntimeError("every buffer holds an input that has not been taken yet")
        i = self.head
        with torch.cuda.stream(self.copy_stream):
            if self.used[i]:
                self.copy_stream.wait_event(self.free[i])
            self.bufs[i].copy_(host, non_blocking=True)
            self.ready[i].record(self.copy_stream)
        self.head = (i + 1) % len(self.bufs)
        self.pending += 1

    def get(self, stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
        """The oldest input, made visible to `stream` (default: the current stream).  The
        buffer returns to the pool when release() is called after the step that reads it
        has been queued."""
        if self.pending == 0:
            raise RuntimeError("no input has been put")
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        i = self.tail
        s.wait_event(self.ready[i])
        self._last = (i, s)
        self.tail = (i + 1) % len(self.bufs)
        self.pending -= 1
        return self.bufs[i]

    def release(self):
        """Mark the buffer handed out last as reusable once the work queued so far on its
        stream has finished."""
        i, s = self._last
        self.free[i].record(s)
        self.used[i] = True
