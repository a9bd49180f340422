"""Integer-pipe microbenchmarks behind the roofline denominators.

    python -m paper_2404_10404_b300.microbench

Times independent 32-bit multiply-add chains (mad.lo, mad.hi) and chained
Montgomery products on every SM of cuda:0, and prints one JSON line.
"""
import json

import paper_2404_10404_b300 as S


def main():
    import torch
    torch.cuda.set_device(0)
    st = torch.cuda.current_stream().cuda_stream
    out = {}
    for name, kind, iters in (("mad_lo", 0, 512), ("mad_hi", 1, 512), ("fr_mul", 2, 128),
                              ("fr_mul_inline", 3, 128), ("mad_wide", 4, 512), ("fr_mul_wide", 5, 128),
                              ("fr_mul_check", 6, 64), ("fr_mac_512", 7, 128), ("fr_sqr", 8, 128),
                              ("fr_mac_512_karatsuba", 9, 128), ("fr_mac_check", 10, 256),
                              ("fr_mul_karatsuba", 11, 128), ("fr_mul_karatsuba_check", 12, 256)):
        ms, ops = S.microbench(kind, 148 * 8, 256, iters, st)
        out[name] = {"ms": ms, "ops": ops, "per_s": ops / (ms / 1e3)}
    # the product rate at the occupancy of the prover kernels (1 and 2 CTAs of 256 per SM)
    for name, blocks in (("fr_mul_1cta_per_sm", 148), ("fr_mul_2cta_per_sm", 296)):
        ms, ops = S.microbench(2, blocks, 256, 512, st)
        out[name] = {"ms": ms, "ops": ops, "per_s": ops / (ms / 1e3)}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
