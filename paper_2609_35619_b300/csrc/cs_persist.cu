// cs_persist.cu -- saving a resident scene to a file and loading it back
// (cs_scene_save / cs_scene_load), so that a process can resume with the
// repacked, Morton-ordered scene without rebuilding it.
//
// File layout (host byte order): a fixed header (magic, version, the
// scene's counts and layout parameters, and the byte offset of every device
// array inside the scene's one allocation), then that allocation byte for
// byte, then the appearance array of the render path when the scene has one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <vector>

#include "cs_internal.cuh"

namespace cs {
namespace {

constexpr char kFileMagic[8] = {'C', 'S', 'B', '3', '0', '0', 'S', 'C'};
constexpr uint32_t kFileVersion = 1;

struct FileHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    int64_t n_input, n_kept, n_grid, n_large, n_invalid;
    int64_t blob_bytes;       // the scene's device allocation
    int64_t app_bytes;        // the appearance array (0: none)
    int32_t nchunks, large_chunk0, n_gauss, nnodes[kLevels];
    float chunk_extent, sigma_tier, pad_abs, bb_lo[3], bb_hi[3];
    // byte offsets inside the allocation
    int64_t off_chead, off_nodes[kLevels], off_smax, off_index, off_slot;
};
// the on-disk header: 192 bytes, off_slot last
static_assert(sizeof(FileHeader) == 192 && offsetof(FileHeader, off_slot) == 184, "scene file header layout");

struct File {
    FILE *f = nullptr;
    ~File() { if (f) fclose(f); }
};

int64_t offset_of(const void *p, const void *base) {
    return p ? (int64_t)((const char *)p - (const char *)base) : -1;
}

}  // namespace
}  // namespace cs

using namespace cs;

extern "C" {

cs_status cs_scene_save(const cs_scene *scene, const char *path, void *stream) {
    cs_status st = check_scene(scene);
    if (st != CS_OK) return st;
    if (!path || !*path) return invalid("path is empty");
    const Scene *sc = reinterpret_cast<const Scene *>(scene);
    if (sc->nblocks != 1) return invalid("internal: a scene is one device allocation");
    int dev = -1;
    CS_CUDA(cudaGetDevice(&dev));
    if (dev != sc->device) return invalid("the scene's device must be the current device");
    const SceneDev &d = sc->dev;
    const void *base = sc->blocks[0];
    FileHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kFileMagic, sizeof(h.magic));
    h.version = kFileVersion;
    h.header_bytes = (uint32_t)sizeof(FileHeader);
    h.n_input = sc->n_input;
    h.n_kept = sc->n_kept;
    h.n_grid = sc->n_grid;
    h.n_large = sc->n_large;
    h.n_invalid = sc->n_invalid;
    h.blob_bytes = sc->device_bytes;
    h.app_bytes = sc->app ? (int64_t)sizeof(float4) * std::max(d.nchunks, 1) * kChunk : 0;
    h.nchunks = d.nchunks;
    h.large_chunk0 = d.large_chunk0;
    h.n_gauss = d.n_gauss;
    for (int l = 0; l < kLevels; ++l) {
        h.nnodes[l] = d.nnodes[l];
        h.off_nodes[l] = offset_of(d.nodes[l], base);
    }
    h.chunk_extent = d.chunk_extent;
    h.sigma_tier = d.sigma_tier;
    h.pad_abs = d.pad_abs;
    for (int k = 0; k < 3; ++k) {
        h.bb_lo[k] = d.bb_lo[k];
        h.bb_hi[k] = d.bb_hi[k];
    }
    h.off_chead = offset_of(d.chead, base);
    h.off_smax = offset_of(d.smax, base);
    h.off_index = offset_of(d.index, base);
    h.off_slot = offset_of(d.slot_of, base);
    std::vector<char> blob((size_t)h.blob_bytes), app((size_t)h.app_bytes);
    cudaStream_t s = (cudaStream_t)stream;
    if (h.blob_bytes > 0) CS_CUDA(cudaMemcpyAsync(blob.data(), base, blob.size(), cudaMemcpyDeviceToHost, s));
    if (h.app_bytes > 0) CS_CUDA(cudaMemcpyAsync(app.data(), sc->app, app.size(), cudaMemcpyDeviceToHost, s));
    CS_CUDA(cudaStreamSynchronize(s));
    File out;
    out.f = fopen(path, "wb");
    if (!out.f) return invalid("cannot open the file for writing");
    if (fwrite(&h, sizeof(h), 1, out.f) != 1 || (blob.size() && fwrite(blob.data(), blob.size(), 1, out.f) != 1) ||
        (app.size() && fwrite(app.data(), app.size(), 1, out.f) != 1))
        return invalid("writing the scene file failed");
    if (fclose(out.f) != 0) {
        out.f = nullptr;
        return invalid("writing the scene file failed");
    }
    out.f = nullptr;
    return CS_OK;
}

cs_status cs_scene_load(const char *path, void *stream, cs_scene **out) {
    if (!out) return invalid("out is NULL");
    *out = nullptr;
    if (!path || !*path) return invalid("path is empty");
    File in;
    in.f = fopen(path, "rb");
    if (!in.f) return invalid("cannot open the scene file");
    FileHeader h;
    if (fread(&h, sizeof(h), 1, in.f) != 1) return invalid("not a scene file (short header)");
    if (memcmp(h.magic, kFileMagic, sizeof(h.magic)) != 0) return invalid("not a scene file (magic)");
    if (h.version != kFileVersion || h.header_bytes != sizeof(FileHeader))
        return invalid("scene file of another format version");
    // the layout must be self-consistent before anything is allocated
    const int64_t blob = h.blob_bytes;
    auto inside = [&](int64_t off, int64_t bytes) { return off >= 0 && bytes >= 0 && off + bytes <= blob; };
    const int64_t nk = std::max<int64_t>(h.n_kept, 1);
    bool ok = blob > 0 && blob <= ((int64_t)1 << 40) && h.n_kept >= 0 && h.n_kept == h.n_gauss &&
              h.n_grid >= 0 && h.n_large >= 0 && h.n_grid + h.n_large == h.n_kept && h.nchunks >= 0 &&
              h.large_chunk0 >= 0 && h.large_chunk0 <= h.nchunks &&
              (int64_t)sizeof(ChunkBlock) * std::max(h.nchunks, 1) <= blob &&
              inside(h.off_chead, (int64_t)sizeof(NodeBox) * std::max(h.nchunks, 1)) &&
              inside(h.off_smax, 4 * nk) && inside(h.off_index, 4 * nk) && inside(h.off_slot, 4 * nk) &&
              h.n_gauss <= (int64_t)h.nchunks * kChunk &&
              (h.app_bytes == 0 || h.app_bytes == (int64_t)sizeof(float4) * std::max(h.nchunks, 1) * kChunk);
    // the node levels of the implicit fan-out-32 tree over the chunks
    for (int l = 0, m = h.nchunks; l < kLevels && ok; ++l) {
        m = (m + 31) / 32;
        ok = h.nnodes[l] == std::max(m, h.nchunks > 0 ? 1 : 0) &&
             inside(h.off_nodes[l], (int64_t)sizeof(NodeBox) * std::max(h.nnodes[l], 1));
    }
    if (!ok) return invalid("scene file with an inconsistent layout");
    std::vector<char> data((size_t)blob), app((size_t)h.app_bytes);
    if (fread(data.data(), data.size(), 1, in.f) != 1) return invalid("scene file truncated");
    if (app.size() && fread(app.data(), app.size(), 1, in.f) != 1) return invalid("scene file truncated");
    // the export reads slot_of[p] as a slot address: every value must name a slot
    {
        const int32_t *slot = reinterpret_cast<const int32_t *>(data.data() + h.off_slot);
        const int64_t nslots = (int64_t)h.nchunks * kChunk;
        for (int64_t p = 0; p < h.n_gauss; ++p)
            if (slot[p] < 0 || slot[p] >= nslots) return invalid("scene file with a slot index out of range");
    }

    Scene *sc = new Scene();
    auto fail = [&](cs_status e) {
        for (int i = 0; i < sc->nblocks; ++i) cudaFree(sc->blocks[i]);
        if (sc->app) cudaFree(sc->app);
        delete sc;
        return e;
    };
    cudaError_t e = cudaGetDevice(&sc->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sc->num_sms, cudaDevAttrMultiProcessorCount, sc->device);
    if (e != cudaSuccess) return fail(cuda_fail(e, "device query"));
    void *base = nullptr;
    e = cudaMalloc(&base, (size_t)blob);
    if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? (set_error("scene allocation failed"), CS_ERR_NO_MEMORY)
                                                                     : cuda_fail(e, "cudaMalloc(scene)"));
    sc->blocks[sc->nblocks++] = base;
    if (app.size()) {
        e = cudaMalloc(&sc->app, app.size());
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(appearance)"));
    }
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemcpyAsync(base, data.data(), data.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && app.size()) e = cudaMemcpyAsync(sc->app, app.data(), app.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host buffers are released on return
    if (e != cudaSuccess) return fail(cuda_fail(e, "uploading the scene"));
    char *b = static_cast<char *>(base);
    SceneDev &d = sc->dev;
    d.blocks = reinterpret_cast<const ChunkBlock *>(b);
    d.chead = reinterpret_cast<const NodeBox *>(b + h.off_chead);
    for (int l = 0; l < kLevels; ++l) {
        d.nodes[l] = reinterpret_cast<const NodeBox *>(b + h.off_nodes[l]);
        d.nnodes[l] = h.nnodes[l];
    }
    d.smax = reinterpret_cast<const float *>(b + h.off_smax);
    d.index = reinterpret_cast<const int32_t *>(b + h.off_index);
    d.slot_of = reinterpret_cast<const int32_t *>(b + h.off_slot);
    d.n_gauss = h.n_gauss;
    d.nchunks = h.nchunks;
    d.large_chunk0 = h.large_chunk0;
    d.chunk_extent = h.chunk_extent;
    d.sigma_tier = h.sigma_tier;
    d.pad_abs = h.pad_abs;
    for (int k = 0; k < 3; ++k) {
        d.bb_lo[k] = h.bb_lo[k];
        d.bb_hi[k] = h.bb_hi[k];
    }
    sc->n_input = h.n_input;
    sc->n_kept = h.n_kept;
    sc->n_grid = h.n_grid;
    sc->n_large = h.n_large;
    sc->n_invalid = h.n_invalid;
    sc->device_bytes = blob;
    sc->magic = kSceneMagic;
    *out = reinterpret_cast<cs_scene *>(sc);
    return CS_OK;
}

}  // extern "C"
