"""The hub-net threshold rule, restated on the host for the GPU tests: the
smallest size on the ladder 512 * 2^(k/2) (k < 24) such that the nets larger
than it, at the first round's bitmap width (every color of round 0 is at most
max(maxnet - 1, 0) + C * Q, plus the C + 2 spare colors of the width, rounded
up to 128-color groups), take at most half the L2 cache."""
import numpy as np

LADDER = [(724 if k & 1 else 512) << (k >> 1) for k in range(24)]
NONE = 2**31 - 1


def first_round_words(maxnet: int, chunk: int, waves: int) -> int:
    ncol = max(maxnet - 1, 0) + chunk * waves + chunk + 2
    return ((ncol + 31) // 32 + 3) & ~3


def expected_threshold(net_sizes, chunk: int, waves: int, l2_bytes: int) -> int:
    sizes = np.asarray(net_sizes, dtype=np.int64)
    if sizes.size == 0:
        return NONE
    words = first_round_words(int(sizes.max()), chunk, waves)
    H = NONE
    for k in range(len(LADDER) - 1, -1, -1):
        if int((sizes > LADDER[k]).sum()) * words * 4 > l2_bytes // 2:
            break
        H = LADDER[k]
    return H


def check(st, net_sizes, chunk=64, waves=16):
    """The call's reported threshold and hub count follow the rule."""
    import torch
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    sizes = np.asarray(net_sizes, dtype=np.int64)
    H = expected_threshold(sizes, chunk, waves, l2)
    assert st["hub_threshold"] == H, (st["hub_threshold"], H)
    assert st["hubs"] == (int((sizes > H).sum()) if H != NONE else 0)
    return H
