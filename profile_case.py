"""Run one workload's sort twice (a warm-up and the captured one) so that a
profiler can capture the second sort's kernel launches.

    python profile_case.py VARIANT WORKLOAD

VARIANT: melded | divergent.  WORKLOAD: cfg1 (4096 uint32 keys, one block),
oem4096 (the same keys through the single-block odd-even merge sort network),
oem26 (2^26 uint32 keys through that network in buckets of 4096, one block each),
SB1 | SB4 | SB1-R | SB4-R (the synthetic divergent kernels, 1216 blocks),
kv24 (2^24 uint32 key-value pairs), f32 (2^26 float32 keys),
pcm26 (PCM of 2^26 uint32 keys in buckets of 4096: one bucket-sort launch and
105 merge-split layer launches per sort, then one gather launch).

The whole-array workloads (cfg1, kv24, f32) run the array's plan one launch
at a time in plan order (darm_sort_profile): the same kernels, launch shapes
and comparators as a sort, but not the split schedule that sorts of 2^22
elements or more use (two halves on two streams, then the final stage), so
that a launch's index in the capture names the same pass of every sort.
"""
import sys

import numpy as np
import torch

import paper_2107_05681_gb300 as darm
import synth


def main(variant="melded", workload="kv24"):
    darm.init(0)
    if workload.startswith("SB"):
        data = torch.from_numpy(synth.uniform_u32(0xDA2C0007, 1024 * 152 * 8)).cuda()
        for _ in range(2):
            d2 = data.clone()
            darm.sb_run(workload, d2, 16, 32, variant=variant)
        torch.cuda.synchronize()
        print("ok", darm.launch_count())
        return
    if workload in ("oem4096", "oem26"):
        keys = synth.cfg1_keys() if workload == "oem4096" else synth.uniform_u32(0xDA2C0006, 1 << 26)
        K = torch.from_numpy(keys).cuda()
        for _ in range(2):
            K2 = K.clone()
            darm.oddeven_sort_buckets(K2, bucket=4096, variant=variant)
        torch.cuda.synchronize()
        print("ok", darm.launch_count())
        return
    if workload == "pcm26":
        K = torch.from_numpy(synth.uniform_u32(0xDA2C0008, 1 << 26)).cuda()
        S = torch.empty_like(K)
        for _ in range(2):
            K2 = K.clone()
            darm.pcm_sort(K2, bucket=4096, scratch_keys=S, variant=variant)
        torch.cuda.synchronize()
        print("ok", darm.launch_count())
        return
    if workload == "kv24":
        k, v = synth.cfg2_kv()
    elif workload == "cfg1":
        k, v = synth.cfg1_keys(), None
    else:
        k, v = synth.cfg3_f32(), None
    K = torch.from_numpy(k).cuda()
    V = torch.from_numpy(v).cuda() if v is not None else None
    for _ in range(2):
        K2 = K.clone()
        V2 = V.clone() if V is not None else None
        darm.sort_profile(K2, V2, variant=variant)
    torch.cuda.synchronize()
    print("ok", darm.launch_count())


if __name__ == "__main__":
    main(*sys.argv[1:3])
