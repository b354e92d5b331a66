// autotune.cu -- choice of the step kernel of a single-instance context by measurement
// (block_cells = LBM_BLOCK_AUTO).
//
// Candidates: the tile kernel over fluid cells (128 cells a block) and, where the layout
// and box allow it, the TMA brick kernel (256 cells a block).  The two give bit-identical
// states, so the choice changes only the time a step takes.  Each candidate runs on a
// temporary copy of the instance (same descriptor, own memory), so the context's own state
// is untouched: warm-up steps, then the time of a fixed number of steps by CUDA events on
// the context's stream, best of two.  A candidate that cannot be had (no memory for the
// copy, a failed launch, a brick copy past its wait limit) is dropped; the tiles are the
// fallback.
//
// Choices are kept per (box, fluid cells, storage, collision, wall, layout, device) for the
// life of the process and, when LBM_AUTOTUNE_CACHE names a file, in that file: one line per
// measurement, "<key>\t<block_cells>\t<ms per step, tiles>\t<ms per step, bricks>", later
// lines overriding earlier ones.  A key found there is not measured again.
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>

#include "batch.h"

namespace lbm {
namespace {

struct Tuned {
    int block = 0;
    double ms[2] = {0.0, 0.0};  // ms per step: tiles, bricks (0 = not measured)
};

std::mutex g_mu;
std::map<std::string, Tuned> g_cache;
std::string g_loaded;  // the cache file last read into g_cache

std::string cache_file()
{
    const char *p = std::getenv("LBM_AUTOTUNE_CACHE");
    return p ? std::string(p) : std::string();
}

void read_file(const std::string &path)
{
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        std::istringstream ls(line);
        std::string key;
        Tuned t;
        if (!std::getline(ls, key, '\t')) continue;
        if (!(ls >> t.block >> t.ms[0] >> t.ms[1])) continue;
        if (t.block != kTileApiCells && t.block != kBrickCells) continue;
        g_cache[key] = t;
    }
}

void append_file(const std::string &path, const std::string &key, const Tuned &t)
{
    std::ofstream f(path, std::ios::app);
    if (!f) return;  // an unwritable cache only costs a measurement next time
    f << key << '\t' << t.block << '\t' << t.ms[0] << '\t' << t.ms[1] << '\n';
}

std::string make_key(const lbm_desc &d, long long n_fluid)
{
    int dev = 0, sms = 0;
    cudaDeviceProp prop{};
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetDeviceProperties(&prop, dev);
    std::ostringstream k;
    k << d.nx << 'x' << d.ny << 'x' << d.nz << " fluid=" << n_fluid << " storage=" << d.storage
      << " collision=" << d.collision << " wall=" << d.wall << " layout=" << d.layout << " gpu=" << prop.name << '/'
      << sms;
    return k.str();
}

bool bricks_allowed(const lbm_desc &d)
{
    return d.layout == LBM_LAYOUT_AB && d.nx % kBrickX == 0 && d.ny % kBrickY == 0 && d.nz % kBrickZ == 0 &&
           d.nx / kBrickX <= 1024 && d.ny / kBrickY <= 2048 && d.nz / kBrickZ <= 2048;
}

// Milliseconds per step of the step kernel block_cells on a copy of the instance d, or a
// negative value when the candidate cannot run.
double time_candidate(const lbm_desc &d0, cudaStream_t s, int block_cells, long long n_fluid)
{
    lbm_desc d = d0;
    d.block_cells = block_cells;
    Batch t;
    std::unique_ptr<Instance> in;
    if (t.init(s, d.storage, d.collision, d.layout) != LBM_OK) return -1.0;
    if (Batch::make_instance(d, s, &in) != LBM_OK) return -1.0;
    if (t.add(std::move(in)) != LBM_OK || t.set_block(block_cells) != LBM_OK || t.prepare() != LBM_OK) return -1.0;
    if (t.block_cells() != block_cells) return -1.0;
    // about 2e8 cell updates per timing, 10 to 200 steps
    const long long n = std::max(10ll, std::min(200ll, 200000000ll / std::max(1ll, n_fluid)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return -1.0;
    }
    double best = -1.0;
    bool ok = t.init_equilibrium(0) == LBM_OK && t.step(5) == LBM_OK && t.fetch_sums() == LBM_OK;
    for (int rep = 0; rep < 2 && ok; ++rep) {
        ok = cudaEventRecord(e0, t.stream()) == cudaSuccess && t.step(n) == LBM_OK &&
             cudaEventRecord(e1, t.stream()) == cudaSuccess && t.fetch_sums() == LBM_OK;
        float ms = 0.0f;
        if (ok) ok = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        if (ok && (best < 0 || ms / n < best)) best = ms / n;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ok ? best : -1.0;
}

}  // namespace

lbm_status autotune_block(Batch &b, const lbm_desc &d, cudaStream_t s)
{
    if (b.size() != 1) return b.set_block(kTileApiCells);
    const long long n_fluid = b.at(0).geo.n_fluid;
    const std::string key = make_key(d, n_fluid);
    const std::string file = cache_file();
    Tuned t;
    bool found = false;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!file.empty() && file != g_loaded) {
            read_file(file);
            g_loaded = file;
        }
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            t = it->second;
            found = true;
        }
    }
    if (!found) {
        t.ms[0] = time_candidate(d, s, kTileApiCells, n_fluid);
        t.ms[1] = bricks_allowed(d) ? time_candidate(d, s, kBrickCells, n_fluid) : -1.0;
        t.block = (t.ms[1] > 0 && (t.ms[0] <= 0 || t.ms[1] < t.ms[0])) ? kBrickCells : kTileApiCells;
        for (double &m : t.ms) m = std::max(m, 0.0);
        set_error("");  // a dropped candidate is not an error of the context
        std::lock_guard<std::mutex> lk(g_mu);
        g_cache[key] = t;
        if (!file.empty()) append_file(file, key, t);
    }
    b.set_tuning(found ? 2 : 1, t.ms[0], t.ms[1]);
    return b.set_block(t.block);
}

}  // namespace lbm
