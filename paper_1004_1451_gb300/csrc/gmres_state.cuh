// Layout of the small FP64 state of flexible GMRES kept on the device: the two
// Gram-Schmidt coefficient vectors, the rotated Hessenberg R (column-major m x m), the
// Givens cosines/sines, the right-hand side g, the solution y and a few scalars.
#pragma once

namespace bamg {

constexpr int GMRES_MMAX = 256;

struct GmresLayout {
    int h1, h2, R, cs, sn, g, y, nrm2, est, hn, rhn, total;  // est, hn adjacent (read together)
    __host__ __device__ explicit GmresLayout(int m) {
        int o = 0;
        h1 = o;
        o += m + 1;
        h2 = o;
        o += m + 1;
        R = o;
        o += m * m;
        cs = o;
        o += m;
        sn = o;
        o += m;
        g = o;
        o += m + 1;
        y = o;
        o += m;
        nrm2 = o++;
        est = o++;
        hn = o++;
        rhn = o++;  // 1 / hn
        total = o;
    }
};

}  // namespace bamg
