"""Host side of the t-slab domain decomposition (Sec. 6) across processes, one rank per
GPU: face exchange with the two t-neighbours and global sums, each bounded by a
deadline. The faces are whatever the caller packs (the library packs spin-projected
boundary slices, 12 reals per face site); this module only moves them. A message that
does not arrive in time raises HaloTimeout (code ERR_TIMEOUT = -8, as in the C ABI)
instead of blocking: a rank that died or stopped sending is reported to the caller,
which then tears the process group down (after a timeout the backend may have closed
the connection, so no further collective is attempted on that group).

Rank r holds global time-slices [r LT/P, (r+1) LT/P); its next rank is r+1 (mod P), its
previous rank r-1 (mod P). Each exchange sends the rank's first slice to the previous
rank (which uses it for its forward t-hops) and its last slice to the next rank (backward
t-hops). With one rank the faces are its own (periodic wrap), copied without messages."""
import datetime
import time

import torch
import torch.distributed as dist

ERR_TIMEOUT = -8
TAG_TO_PREV, TAG_TO_NEXT = 101, 102


class HaloTimeout(RuntimeError):
    def __init__(self, what, seconds):
        super().__init__(f"ERR_TIMEOUT: {what} not complete after {seconds:.3f} s")
        self.code = ERR_TIMEOUT


class HaloExchange:
    def __init__(self, timeout_s=1.0, group=None):
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.next = (self.rank + 1) % self.world
        self.prev = (self.rank - 1) % self.world
        self.timeout_s = timeout_s

    def _wait(self, works, what):
        deadline = time.monotonic() + self.timeout_s
        for w in works:
            left = deadline - time.monotonic()
            if left <= 0:
                raise HaloTimeout(what, self.timeout_s)
            try:
                done = w.wait(timeout=datetime.timedelta(seconds=left))
            except RuntimeError as e:  # the backend reports its own timeout as an error
                if "timed out" in str(e).lower() or "timeout" in str(e).lower():
                    raise HaloTimeout(what, self.timeout_s) from e
                raise
            if done is False:
                raise HaloTimeout(what, self.timeout_s)

    def exchange(self, to_prev, to_next):
        """Send `to_prev` (first slice) to the previous rank and `to_next` (last slice) to
        the next rank; return (from_next, from_prev): the next rank's first slice and the
        previous rank's last slice."""
        if self.world == 1:
            return to_prev.clone(), to_next.clone()
        from_next = torch.empty_like(to_prev)
        from_prev = torch.empty_like(to_next)
        works = [dist.irecv(from_next, src=self.next, tag=TAG_TO_PREV, group=self.group),
                 dist.irecv(from_prev, src=self.prev, tag=TAG_TO_NEXT, group=self.group),
                 dist.isend(to_prev.contiguous(), dst=self.prev, tag=TAG_TO_PREV, group=self.group),
                 dist.isend(to_next.contiguous(), dst=self.next, tag=TAG_TO_NEXT, group=self.group)]
        self._wait(works, "halo exchange")
        return from_next, from_prev

    def allreduce(self, x):
        """Sum of x over the ranks, in place."""
        if self.world > 1:
            self._wait([dist.all_reduce(x, group=self.group, async_op=True)], "allreduce")
        return x
