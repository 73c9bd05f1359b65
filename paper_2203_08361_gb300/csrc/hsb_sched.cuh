// hsb_sched.cuh -- tile order of the one-step kernels (host and device).
#pragma once

namespace hsb {

// Tile t -> (row block mb, replica block rb).  The replica blocks are cut
// into bands of `band` blocks (the last band may be narrower) taken one after
// another; inside a band the tiles run row block by row block with the band's
// replica blocks fastest.  The CTAs running at one time then share the J rows
// of a few row blocks, and the band's S rows, which every row block reads,
// stay in L2 while the row blocks pass.
__host__ __device__ __forceinline__ void tile_coords(int t, int nmb, int nrb, int band, int &mb,
                                                     int &rb)
{
    const int per = nmb * band;
    const int k = t / per;
    const int rem = t - k * per;
    const int w = band < nrb - k * band ? band : nrb - k * band;
    mb = rem / w;
    rb = k * band + (rem - mb * w);
}

}  // namespace hsb
