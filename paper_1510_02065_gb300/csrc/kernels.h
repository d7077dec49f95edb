// kernels.h -- host-side launchers of the device kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace rlt2 {

struct DevStatus;

// Geometry of the tile store of D.  Tile t = ((i*N + j)*(N-1) + k')*(N-1) + n'
// holds the submatrix D_ijkn: its N-2 rows are the facilities p not in {i,k}
// (ascending) and its columns are indexed by the location q itself, W =
// round_up(N, 4) of them; columns j and n (and q >= N) carry no coefficient.
// Every row starts on a 16-byte boundary and any 4 consecutive locations
// 4c..4c+3 form one aligned 16-byte piece of a row.
struct Geom {
    int N;
    int n;            // N - 2: rows (and coefficients per row) of a tile
    int W;            // row width in ints, round_up(N, 4)
    int TS;           // tile stride, ints (n * W)
    long long tiles;  // N^2 (N-1)^2
};

inline Geom make_geom(int N)
{
    Geom g;
    g.N = N;
    g.n = N - 2;
    g.W = (N + 3) & ~3;
    g.TS = g.n * g.W;
    g.tiles = (long long)N * N * (N - 1) * (N - 1);
    return g;
}

// Per-pass device state shared by the stage kernels.
struct PassState {
    int *z;                  // tile store of D
    int *yS;                 // S of each D-tile concentration (C before its transfer)
    int *yC;                 // reduced C after concentration C->B
    int *x;                  // reduced B
    long long *LB;           // bound
    long long *hist;         // LB after each pass
    int *iter;               // passes completed
    int *stop;               // stopping rule fired
    unsigned *counter;       // work counter of the D->C sweep
    DevStatus *status;
    int hist_cap;
    double ub, min_progress;
    bool pack;               // keys fit the packed reduction
    bool rlt1_only;
};

cudaError_t launch_init(const Geom &g, const PassState &p, const int32_t *F, const int32_t *D,
                        const int32_t *Blin, long long lb_const, cudaStream_t s);
cudaError_t launch_spread_x(const Geom &g, const PassState &p, cudaStream_t s);
cudaError_t launch_p1(const Geom &g, const PassState &p, const int4 *triples, int ntriples,
                      cudaStream_t s);
cudaError_t launch_dlap(const Geom &g, const PassState &p, int sm_count, cudaStream_t s);
cudaError_t launch_clap(const Geom &g, const PassState &p, cudaStream_t s);
cudaError_t launch_xlap(const Geom &g, const PassState &p, cudaStream_t s);
cudaError_t launch_lap_batch(const int32_t *M, int n, int count, int64_t *S, int32_t *assign,
                             int32_t *u, int32_t *v, int64_t *work, DevStatus *status,
                             cudaStream_t s);

int p1_chunk(int N);                    // locations per CTA of the fused pass over D
size_t p1_smem_bytes(int N, int JC);    // its dynamic shared memory
}  // namespace rlt2
