"""One FP32 volume-operator matvec (K1, five FFT passes) on the head-size
extended grid (128 x 128 x 112, body 96 x 96 x 112 at 2 mm), bracketed by
cudaProfilerStart/Stop so that an ncu capture started with
--profile-from-start off records exactly that matvec's kernels:

    ncu --profile-from-start off --set full --clock-control none \\
        -k regex:"k_(xfwd|ypass|zmul|xinv)" -c 5 -o prof \\
        python -m paper_2206_12409_gb300.profile_conv
"""
import sys

import torch

from paper_2206_12409_gb300 import inputs as I
from paper_2206_12409_gb300 import vsie as V


def main(p=1):
    g, er, sg = I.layered_head_phantom()
    ctx = V.vsie_create(V.make_grid(g.n, g.h, g.origin), er, sg, 298e6,
                        V.make_options(ext_n=(128, 128, 112), ext_offset=(16, 16, 0), max_rhs=p,
                                       precisions=1 << V.VSIE_C64))
    N = V.vsie_sizes(ctx)[0]
    X = torch.randn((p, N), dtype=torch.complex64, device="cuda")
    Y = torch.empty_like(X)
    for _ in range(3):
        V.vsie_matvec(ctx, p, X.data_ptr(), N, Y.data_ptr(), N, V.VSIE_C64)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    V.vsie_matvec(ctx, p, X.data_ptr(), N, Y.data_ptr(), N, V.VSIE_C64)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    V.vsie_destroy(ctx)
    print("done")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 1)
