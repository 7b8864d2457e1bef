// Fused leap-frog step on TMA-staged (r, phi, z) tiles (zda_tile.cu).
#pragma once
#include <cuda.h>
#include "zda_internal.h"

namespace zda {

// Tensor maps of one field buffer ([n_r][n_phi][n_z] complex FP32 per
// component, seen as FP32 with dims (2 n_z, n_phi, n_r)): the E slab and H
// slab of a tile at one radius, and the one-row boxes that fetch the
// phi-wrapped halo rows.
struct TileMaps {
    CUtensorMap e[3], ew[3], h[3], hw[3];
};

// Tensor maps for the E tile kernel (split step, E half): the tile's own E
// box, the H slab (one row and two z-cells more below), the wrapped H row.
struct TileEMaps {
    CUtensorMap eo[3], h[3], hw[3];
};

// Tensor maps for the H tile kernel (split step, H half): the E slab (one row
// and two z-cells more above), the wrapped E row, the tile's own H box.
struct TileHMaps {
    CUtensorMap e[3], ew[3], ho[3];
};

struct TileParams {
    StepParams p;                 // tables, E-side CPML (updated in place), density, source, DFT history
    float2 *oE[3], *oH[3];        // destination buffer: E^{n+1}, H^{n+1/2}
    const float2 *psH_in[4];      // H-side CPML auxiliaries at n-1/2: hr_z, hp_z, hp_r, hz_r
    float2 *psH_out[4];           // ... at n+1/2 (the other set)
    int *err;                     // error word: a bounded wait gave up
    int wait_limit;               // polls of the tile's mbarrier before giving up
    int inject_timeout;           // tests: thread 0 first waits on a barrier that nothing completes
};

// tile shapes compiled: tj in {4, 8, 16} phi rows, 32 z-cells; each thread block streams
// over a range of radii (n_rchunks ranges per tile column)
bool tile_shape_ok(int tj);
constexpr int TILE_KZ = 32;
size_t tile_smem_bytes(int tj);
int tile_blocks_per_sm(int tj);
int tile_auto_rchunks(int tj, int nr, int nphi, int nz, int sms);
// false if the driver's tensor-map encoder is unavailable or refuses the layout
bool encode_tile_maps(TileMaps *m, float2 *const E[3], float2 *const H[3], int nr, int nphi, int nz, int tj,
                      const char **why);
cudaError_t launch_tile_step(const TileMaps &m, const TileParams &tp, int n, int tj, int n_rchunks, cudaStream_t s);

// E half of the split step on TMA-staged tiles of tj in {8, 16, 32} phi rows x 32 z-cells,
// updating E in place; TileParams::oE = the field buffer's E, the H-side members unused
bool tile_e_shape_ok(int tj);
size_t tile_e_smem_bytes(int tj);
int tile_e_auto_rchunks(int tj, int nr, int nphi, int nz, int sms);
bool encode_tile_e_maps(TileEMaps *m, float2 *const E[3], float2 *const H[3], int nr, int nphi, int nz, int tj,
                        const char **why);
cudaError_t launch_tile_e(const TileEMaps &m, const TileParams &tp, int n, int tj, int n_rchunks, cudaStream_t s);
// H half of the split step on the same tiles (shapes and radius ranges as the E tile kernel),
// updating H and the H-side CPML auxiliaries in place; TileParams::oH = the field buffer's H
bool encode_tile_h_maps(TileHMaps *m, float2 *const E[3], float2 *const H[3], int nr, int nphi, int nz, int tj,
                        const char **why);
cudaError_t launch_tile_h(const TileHMaps &m, const TileParams &tp, int tj, int n_rchunks, cudaStream_t s);

}  // namespace zda
