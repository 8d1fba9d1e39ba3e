"""Distributed N-D permute over torch.distributed ranks, one GPU each
(include/librearr_dist.h): the library's pack permute, an all-to-all of
equal pieces, and the library's unpack permute.  torch.distributed carries
the exchange (NCCL between GPUs); both local steps are librearr kernels."""
from typing import Sequence

from . import librearr


def dist_permute(out_slab, in_slab, elem_bytes: int, dims: Sequence[int], perm: Sequence[int], group=None,
                 stream=None) -> librearr.DistPlan:
    """out_slab <- this rank's output slab of the global array `dims`
    permuted by `perm` (numpy semantics), given this rank's input slab.
    Input and output are sharded along their slowest axis in equal slabs
    (rank r holds rows [r*n/P, (r+1)*n/P) of that axis).  Both slabs are
    CUDA tensors of at least plan.slab_bytes; the call enqueues on `stream`
    (the current stream by default) and returns the plan."""
    import torch
    import torch.distributed as dist

    if not (in_slab.is_cuda and out_slab.is_cuda):
        raise ValueError("dist_permute works on CUDA tensors (the pack and unpack are device kernels)")
    nranks = dist.get_world_size(group)
    plan = librearr.dist_permute_plan(elem_bytes, dims, perm, nranks)
    for t, what in ((in_slab, "in_slab"), (out_slab, "out_slab")):
        if t.numel() * t.element_size() < plan.slab_bytes:
            raise ValueError(f"{what} holds fewer than {plan.slab_bytes} bytes")
    s = stream if stream is not None else torch.cuda.current_stream(in_slab.device)
    if not plan.exchange:
        librearr.dist_permute_pack(out_slab, in_slab, plan, elem_bytes, s)
        return plan
    send = torch.empty(plan.slab_bytes, dtype=torch.uint8, device=in_slab.device)
    recv = torch.empty_like(send)
    with torch.cuda.stream(s):
        librearr.dist_permute_pack(send, in_slab, plan, elem_bytes, s)
        dist.all_to_all_single(recv, send, group=group)
        librearr.dist_permute_unpack(out_slab, recv, plan, elem_bytes, s)
        # the buffers must outlive the kernels and the collective on s
        send.record_stream(s)
        recv.record_stream(s)
    return plan
