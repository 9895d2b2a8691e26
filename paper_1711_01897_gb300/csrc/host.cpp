// Host side of the GB300 BEM library: the C ABI of include/bem.h, mesh
// validation and adjacency, quadrature tables, the cluster and block
// cluster trees (Sec. 2.1; Algorithm "H-Matrix Assembly", Sec. 4.1) and the
// orchestration of the device kernels.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/bem.h"
#include "bem_internal.h"
#include "bem_host_internal.h"

#include <atomic>
#include <condition_variable>
#include <unistd.h>
#include <functional>
#include <thread>

using namespace bem;

namespace bem {
int aca_small_cap();
int aca_tiny_max();

static std::mutex g_tune_mu;
static bem_tuning g_tuning{8192, 0, 1};
static bem_quadrature g_quad{0.0, 0.0};

static std::atomic<int64_t> g_launches{0};
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }
}

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

struct CudaFail {
    int code;
};

#define CU(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            g_err = std::string(#call) + ": " + cudaGetErrorString(e_);                   \
            throw CudaFail{e_ == cudaErrorMemoryAllocation ? BEM_E_OOM : BEM_E_CUDA};     \
        }                                                                                 \
    } while (0)

template <class F>
int guarded(F &&f)
{
    try {
        g_err.clear();
        return f();
    } catch (const CudaFail &c) {
        return c.code;
    } catch (const std::bad_alloc &) {
        return fail(BEM_E_OOM, "host allocation failed");
    } catch (const std::exception &ex) {
        return fail(BEM_E_ARG, ex.what());
    }
}

// The library's stream-ordered memory pool on the current device.  Freed
// blocks up to kPoolKeep bytes stay in the pool across synchronisations, so
// that meshes, trees and factor pools created one after another reuse them
// instead of mapping fresh memory each time (the device's default pool
// returns everything at every synchronisation).  pool_trim hands the cached
// blocks back, before a large allocation is sized against the free memory.
constexpr uint64_t kPoolKeep = uint64_t(16) << 30;
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;

cudaMemPool_t lib_pool()
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) return it->second;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        cudaDeviceGetDefaultMemPool(&pool, dev);
    } else {
        uint64_t keep = kPoolKeep;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    g_pools[dev] = pool;
    return pool;
}

void pool_trim()
{
    cudaMemPoolTrimTo(lib_pool(), 0);
}

// Pinned host slots of up to kPinSlot bytes for the small readbacks and
// uploads of an assembly (pool header, totals, the ACA job).  They come from
// page-locked chunks that are never returned: freeing page-locked memory
// synchronises the whole device, which would stall every stream (the request
// server frees matrices while other batches run).
constexpr size_t kPinSlot = 256, kPinChunk = 64 * 1024;
std::mutex g_pin_mu;
std::vector<void *> g_pin_free;

void *pinned_slot()
{
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (g_pin_free.empty()) {
        void *chunk = nullptr;
        if (cudaMallocHost(&chunk, kPinChunk) != cudaSuccess) return nullptr;
        for (size_t o = 0; o < kPinChunk; o += kPinSlot) g_pin_free.push_back((char *)chunk + o);
    }
    void *p = g_pin_free.back();
    g_pin_free.pop_back();
    return p;
}

void pinned_release(void *p)
{
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(p);
}

cudaError_t lib_malloc_async(void **p, size_t b, cudaStream_t st)
{
    return cudaMallocFromPoolAsync(p, b, lib_pool(), st);
}

// Device buffer owned by RAII, allocated stream-ordered on its home stream
// from the library's pool and freed on that stream.
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaStream_t home = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() { release(); }
    void release()
    {
        if (p) cudaFreeAsync(p, home);
        p = nullptr;
        bytes = 0;
    }
    void alloc(size_t b, cudaStream_t st = 0)
    {
        release();
        if (b == 0) b = 16;
        home = st;
        cudaError_t e = lib_malloc_async(&p, b, st);
        if (e != cudaSuccess) {
            p = nullptr;
            g_err = "device allocation of " + std::to_string(b) + " bytes failed: " +
                    cudaGetErrorString(e);
            throw CudaFail{e == cudaErrorMemoryAllocation ? BEM_E_OOM : BEM_E_CUDA};
        }
        bytes = b;
    }
    template <class T>
    T *as() const
    {
        return reinterpret_cast<T *>(p);
    }
    template <class T, class A>
    void upload(const std::vector<T, A> &v, cudaStream_t st = 0)
    {
        alloc(v.size() * sizeof(T), st);
        if (!v.empty())
            CU(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    }
};

double now_ms()
{
    return std::chrono::duration<double, std::milli>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// ---------------------------------------------------------------------------
// quadrature tables (derived here, independently of any test code)
// ---------------------------------------------------------------------------

// Gauss-Legendre nodes on [0,1] by Golub-Welsch: eigenvalues of the
// symmetric Jacobi matrix of the Legendre recurrence (off-diagonal
// k / sqrt(4k^2 - 1)), found by cyclic Jacobi rotations; the weights are
// twice the squared first components of the eigenvectors.
void gauss_legendre01(int n, double *x, double *w)
{
    std::vector<double> A(n * n, 0.0), Q(n * n, 0.0);
    for (int i = 0; i < n; ++i) Q[i * n + i] = 1.0;
    for (int k = 1; k < n; ++k) {
        double b = k / std::sqrt(4.0 * k * k - 1.0);
        A[(k - 1) * n + k] = A[k * n + k - 1] = b;
    }
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
        if (off < 1e-34) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) /
                           (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // A <- A J
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // A <- J^T A
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double qkp = Q[k * n + p], qkq = Q[k * n + q];
                    Q[k * n + p] = c * qkp - s * qkq;
                    Q[k * n + q] = s * qkp + c * qkq;
                }
            }
    }
    std::vector<std::pair<double, double>> nw(n);
    for (int i = 0; i < n; ++i) nw[i] = {0.5 * (1.0 + A[i * n + i]), Q[i] * Q[i]};
    std::sort(nw.begin(), nw.end());
    for (int i = 0; i < n; ++i) {
        x[i] = nw[i].first;
        w[i] = nw[i].second;  // 2 v0^2 on [-1,1], halved on [0,1]
    }
}

// Symmetric 6-point rule of degree 4 (Sec. 3.2.1): orbits (a,a,1-2a) and
// (b,b,1-2b).  For given (a,b) the orbit weights follow from the moments of
// 1 and e2 (a 2x2 linear system); (a,b) then solve the moments of e3 and
// e2^2 (1/60, 1/15) by Newton's method with a difference Jacobian.
QuadRule make_rule6()
{
    auto e2 = [](double a) { return 2 * a - 3 * a * a; };
    auto e3 = [](double a) { return a * a * (1 - 2 * a); };
    auto weights = [&](double a, double b, double &W1, double &W2) {
        W1 = (0.25 - e2(b)) / (e2(a) - e2(b));
        W2 = 1.0 - W1;
    };
    auto resid = [&](double a, double b, double r[2]) {
        double W1, W2;
        weights(a, b, W1, W2);
        r[0] = W1 * e3(a) + W2 * e3(b) - 1.0 / 60.0;
        r[1] = W1 * e2(a) * e2(a) + W2 * e2(b) * e2(b) - 1.0 / 15.0;
    };
    double a = 0.44, b = 0.09;
    for (int it = 0; it < 60; ++it) {
        double r[2], ra[2], rb[2], h = 1e-7;
        resid(a, b, r);
        double rap[2], ram[2], rbp[2], rbm[2];
        resid(a + h, b, rap);
        resid(a - h, b, ram);
        resid(a, b + h, rbp);
        resid(a, b - h, rbm);
        for (int c = 0; c < 2; ++c) {
            ra[c] = (rap[c] - ram[c]) / (2 * h);
            rb[c] = (rbp[c] - rbm[c]) / (2 * h);
        }
        double det = ra[0] * rb[1] - rb[0] * ra[1];
        double da = (r[0] * rb[1] - rb[0] * r[1]) / det;
        double db = (ra[0] * r[1] - r[0] * ra[1]) / det;
        a -= da;
        b -= db;
        if (std::fabs(da) + std::fabs(db) < 1e-18) break;
    }
    double W1, W2;
    weights(a, b, W1, W2);
    QuadRule R{};
    R.beta3 = 0.5 / (1.0 - 3.0 * b);
    R.beta3f = (float)R.beta3;
    R.rho21 = (1.0 - 3.0 * b) / (1.0 - 3.0 * a);
    R.rho21f = (float)R.rho21;
    const double orb[2] = {a, b}, ow[2] = {W1 / 3.0, W2 / 3.0};
    int k = 0;
    for (int o = 0; o < 2; ++o) {
        double q = orb[o], r = 1.0 - 2.0 * q;
        const double bary[3][3] = {{q, q, r}, {q, r, q}, {r, q, q}};
        for (int m = 0; m < 3; ++m, ++k) {
            R.s[k] = bary[m][1];
            R.t[k] = bary[m][2];
            R.w[k] = ow[o];
            R.wf[k] = (float)ow[o];
            for (int v = 0; v < 3; ++v) {
                R.wl[k][v] = ow[o] * bary[m][v];
                R.wlf[k][v] = (float)R.wl[k][v];
            }
        }
    }
    return R;
}

// Sauter-Schwab maps of [0,1]^4 onto T^ x T^ (T^ = {0 <= x2 <= x1 <= 1})
// for vertex- (1), edge-adjacent (2) and identical (3) panels, after the
// Erichsen-Sauter scheme (Sec. 3.2.3).  Returns the Jacobian.
double ss_map(int c, int r, double xi, double a, double b, double g, double X[2], double Y[2])
{
    if (c == 3) {
        switch (r) {
        case 0: X[0] = xi; X[1] = xi * (1 - a + a * b); Y[0] = xi * (1 - a * b * g); Y[1] = xi * (1 - a); break;
        case 1: X[0] = xi * (1 - a * b * g); X[1] = xi * (1 - a); Y[0] = xi; Y[1] = xi * (1 - a + a * b); break;
        case 2: X[0] = xi; X[1] = xi * a * (1 - b + b * g); Y[0] = xi * (1 - a * b); Y[1] = xi * a * (1 - b); break;
        case 3: X[0] = xi * (1 - a * b); X[1] = xi * a * (1 - b); Y[0] = xi; Y[1] = xi * a * (1 - b + b * g); break;
        case 4: X[0] = xi * (1 - a * b * g); X[1] = xi * a * (1 - b * g); Y[0] = xi; Y[1] = xi * a * (1 - b); break;
        default: X[0] = xi; X[1] = xi * a * (1 - b); Y[0] = xi * (1 - a * b * g); Y[1] = xi * a * (1 - b * g); break;
        }
        return xi * xi * xi * a * a * b;
    }
    if (c == 2) {
        switch (r) {
        case 0: X[0] = xi; X[1] = xi * a * g; Y[0] = xi * (1 - a * b); Y[1] = xi * a * (1 - b);
            return xi * xi * xi * a * a;
        case 1: X[0] = xi; X[1] = xi * a; Y[0] = xi * (1 - a * b * g); Y[1] = xi * a * b * (1 - g); break;
        case 2: X[0] = xi * (1 - a * b); X[1] = xi * a * (1 - b); Y[0] = xi; Y[1] = xi * a * b * g; break;
        case 3: X[0] = xi * (1 - a * b * g); X[1] = xi * a * b * (1 - g); Y[0] = xi; Y[1] = xi * a; break;
        default: X[0] = xi * (1 - a * b * g); X[1] = xi * a * (1 - b * g); Y[0] = xi; Y[1] = xi * a * b; break;
        }
        return xi * xi * xi * a * a * b;
    }
    if (r == 0) { X[0] = xi; X[1] = xi * a; Y[0] = xi * b; Y[1] = xi * b * g; }
    else { X[0] = xi * b; X[1] = xi * b * g; Y[0] = xi; Y[1] = xi * a; }
    return xi * xi * xi * b;
}

// d = x - y in the case's edge basis (see SingTable).
void ss_coef(int c, const double X[2], const double Y[2], double cf[4])
{
    if (c == 3) { cf[0] = X[0] - Y[0]; cf[1] = X[1] - Y[1]; cf[2] = cf[3] = 0.0; }
    else if (c == 2) { cf[0] = X[0] - Y[0]; cf[1] = X[1]; cf[2] = -Y[1]; cf[3] = 0.0; }
    else { cf[0] = X[0]; cf[1] = X[1]; cf[2] = -Y[0]; cf[3] = -Y[1]; }
}

struct HostSingTable {
    std::vector<double> lap, helm, xy;  // row-major [6][n_lap], [5][n_helm], [4][n_helm]
    int n_lap = 0, n_helm = 0;
};

HostSingTable make_sing_table(int c, const double *x, const double *w)
{
    const int R = c == 3 ? 6 : (c == 2 ? 5 : 2);
    HostSingTable T;
    // Laplace: merge nodes of equal direction c/|c|_max
    std::map<std::array<long long, 4>, int> key_to_idx;
    std::vector<std::array<double, 6>> rows;
    for (int r = 0; r < R; ++r)
        for (int i0 = 0; i0 < NGL; ++i0)
            for (int i1 = 0; i1 < NGL; ++i1)
                for (int i2 = 0; i2 < NGL; ++i2)
                    for (int i3 = 0; i3 < NGL; ++i3) {
                        double X[2], Y[2], cf[4];
                        double J = ss_map(c, r, x[i0], x[i1], x[i2], x[i3], X, Y);
                        ss_coef(c, X, Y, cf);
                        double W = w[i0] * w[i1] * w[i2] * w[i3] * J;
                        double rho = 0.0;
                        for (int q = 0; q < 4; ++q) rho = std::max(rho, std::fabs(cf[q]));
                        std::array<long long, 4> key;
                        double v[4];
                        for (int q = 0; q < 4; ++q) {
                            v[q] = cf[q] / rho;
                            key[q] = std::llround(v[q] * 68719476736.0);  // 2^36
                        }
                        auto it = key_to_idx.find(key);
                        if (it == key_to_idx.end()) {
                            key_to_idx[key] = (int)rows.size();
                            rows.push_back({v[0], v[1], v[2], v[3], W / rho, W / (rho * rho)});
                        } else {
                            rows[it->second][4] += W / rho;
                            rows[it->second][5] += W / (rho * rho);
                        }
                    }
    T.n_lap = (int)rows.size();
    T.lap.assign(6 * T.n_lap, 0.0);
    for (int q = 0; q < T.n_lap; ++q)
        for (int rr = 0; rr < 6; ++rr) T.lap[rr * T.n_lap + q] = rows[q][rr];
    // Helmholtz: eta nodes at xi = 1 (all maps are homogeneous in xi)
    T.n_helm = R * NGL * NGL * NGL;
    T.helm.assign(5 * T.n_helm, 0.0);
    T.xy.assign(4 * T.n_helm, 0.0);
    int q = 0;
    for (int r = 0; r < R; ++r)
        for (int i1 = 0; i1 < NGL; ++i1)
            for (int i2 = 0; i2 < NGL; ++i2)
                for (int i3 = 0; i3 < NGL; ++i3, ++q) {
                    double X[2], Y[2], cf[4];
                    double J = ss_map(c, r, 1.0, x[i1], x[i2], x[i3], X, Y);
                    ss_coef(c, X, Y, cf);
                    for (int rr = 0; rr < 4; ++rr) T.helm[rr * T.n_helm + q] = cf[rr];
                    T.helm[4 * T.n_helm + q] = w[i1] * w[i2] * w[i3] * J;
                    T.xy[0 * T.n_helm + q] = X[0];
                    T.xy[1 * T.n_helm + q] = X[1];
                    T.xy[2 * T.n_helm + q] = Y[0];
                    T.xy[3 * T.n_helm + q] = Y[1];
                }
    return T;
}

// Per-device constant data: rules and singular tables.
struct DeviceConsts {
    QuadRule rule;
    SingTable sing[3];
    DBuf bufs[9];
    int num_sms = 0;
};

std::mutex g_dev_mu;
std::map<int, std::unique_ptr<DeviceConsts>> g_dev;

DeviceConsts &device_consts()
{
    int dev = 0;
    CU(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_dev_mu);
    auto it = g_dev.find(dev);
    if (it != g_dev.end()) return *it->second;
    auto D = std::make_unique<DeviceConsts>();
    D->rule = make_rule6();
    double x[NGL], w[NGL];
    gauss_legendre01(NGL, x, w);
    for (int c = 1; c <= 3; ++c) {
        HostSingTable H = make_sing_table(c, x, w);
        // the singular kernel stages a table of at most 6 * NGL^3 points
        if (H.n_lap > 6 * NGL * NGL * NGL || H.n_helm > 6 * NGL * NGL * NGL)
            throw std::runtime_error("singular quadrature table too large");
        DBuf &bl = D->bufs[3 * (c - 1)], &bh = D->bufs[3 * (c - 1) + 1],
             &bx = D->bufs[3 * (c - 1) + 2];
        bl.upload(H.lap);
        bh.upload(H.helm);
        bx.upload(H.xy);
        CU(cudaStreamSynchronize(0));
        SingTable &S = D->sing[c - 1];
        S.n_lap = H.n_lap;
        S.n_helm = H.n_helm;
        S.lap = bl.as<double>();
        S.helm = bh.as<double>();
        S.xy = bx.as<double>();
        for (int i = 0; i < NGL; ++i) {
            S.xi[i] = x[i];
            S.wxi[i] = w[i];
        }
    }
    CU(cudaDeviceGetAttribute(&D->num_sms, cudaDevAttrMultiProcessorCount, dev));
    DeviceConsts &ref = *D;
    g_dev[dev] = std::move(D);
    return ref;
}

// Device geometry owned by a mesh or an H-matrix.
struct GeomStore {
    DBuf tri, vtx, nrm, area, qp, tq;
    DevGeom g{};
    void build(const double *dV, const int32_t *dT, const int32_t *dperm, int64_t nt,
               const QuadRule &R, cudaStream_t st)
    {
        tri.alloc(3 * nt * sizeof(int32_t), st);
        vtx.alloc(9 * nt * sizeof(double), st);
        nrm.alloc(3 * nt * sizeof(double), st);
        area.alloc(nt * sizeof(double), st);
        qp.alloc(3 * NQ * nt * sizeof(double), st);
        tq.alloc((nt + 31) / 32 * 32 * kTileFields * sizeof(float), st);
        void *const b[6] = {tri.p, vtx.p, nrm.p, area.p, qp.p, tq.p};
        CU(launch_geometry(dV, dT, dperm, nt, R, b, st));
        g.nt = nt;
        g.tri = tri.as<int32_t>();
        g.vtx = vtx.as<double>();
        g.nrm = nrm.as<double>();
        g.area = area.as<double>();
        g.qp = qp.as<double>();
        g.tq = tq.as<float>();
    }
};

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a{};
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// ---------------------------------------------------------------------------
// meshes
// ---------------------------------------------------------------------------
// Allocator whose value-initialisation leaves elements uninitialised: for
// host lists that are written in full right after they are sized.
template <class T>
struct NoInit : std::allocator<T> {
    using value_type = T;
    template <class U>
    struct rebind {
        using other = NoInit<U>;
    };
    NoInit() = default;
    template <class U>
    NoInit(const NoInit<U> &) noexcept {}
    template <class U>
    void construct(U *p) noexcept
    {
        ::new ((void *)p) U;
    }
    template <class U, class... A>
    void construct(U *p, A &&...a)
    {
        ::new ((void *)p) U(std::forward<A>(a)...);
    }
};

struct bem_mesh_s {
    int device = 0;
    int64_t nv = 0, nt = 0;
    std::vector<double> V;
    std::vector<int32_t> T;
    DBuf dV, dT;
    GeomStore geom;
    // touching triangles (sharing >= 1 vertex, itself included): CSR
    std::vector<int64_t, NoInit<int64_t>> adj_ptr;
    std::vector<int32_t, NoInit<int32_t>> adj_tri;
    std::vector<int8_t, NoInit<int8_t>> adj_case;   // shared vertex count 1..3
    int64_t max_touch = 0;
    int hmat_refs = 0;
};

namespace {

// Helper threads of one calling thread, created on its first parallel call
// and reused by the later ones (creating and joining threads for every call
// cost more than the work of most tree-build phases).  Each calling thread
// (the caller's own, a server slot's worker) has its own pool, joined when
// that thread exits.
class TaskPool {
public:
    const pid_t owner = getpid();   // a forked child inherits the object, not the threads
    explicit TaskPool(int helpers)
    {
        for (int i = 0; i < helpers; ++i) workers_.emplace_back([this] { loop(); });
    }
    ~TaskPool()
    {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        wake_.notify_all();
        for (auto &t : workers_) t.join();
    }
    int helpers() const { return (int)workers_.size(); }
    // runs f(task) for task in [0, ntask) on the caller and the helpers
    void run(int64_t ntask, const std::function<void(int64_t)> &f)
    {
        {
            std::lock_guard<std::mutex> lk(mu_);
            job_ = &f;
            ntask_ = ntask;
            next_.store(0);
            busy_ = (int)workers_.size();
            err_.clear();
            ++gen_;
        }
        wake_.notify_all();
        work();
        std::unique_lock<std::mutex> lk(mu_);
        done_.wait(lk, [&] { return busy_ == 0; });
        job_ = nullptr;
        if (!err_.empty()) throw std::runtime_error(err_);
    }

private:
    void work()
    {
        for (;;) {
            const int64_t t = next_.fetch_add(1);
            if (t >= ntask_) return;
            try {
                (*job_)(t);
            } catch (const std::exception &e) {
                std::lock_guard<std::mutex> lk(mu_);
                if (err_.empty()) err_ = e.what();
            }
        }
    }
    void loop()
    {
        uint64_t seen = 0;
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(mu_);
                wake_.wait(lk, [&] { return stop_ || gen_ != seen; });
                if (stop_) return;
                seen = gen_;
            }
            work();
            std::lock_guard<std::mutex> lk(mu_);
            if (--busy_ == 0) done_.notify_all();
        }
    }
    std::vector<std::thread> workers_;
    std::mutex mu_;
    std::condition_variable wake_, done_;
    const std::function<void(int64_t)> *job_ = nullptr;
    int64_t ntask_ = 0;
    std::atomic<int64_t> next_{0};
    int busy_ = 0;
    uint64_t gen_ = 0;
    bool stop_ = false;
    std::string err_;
};

// The calling thread's pool (one per thread, shared by every parallel phase).
TaskPool &thread_pool()
{
    thread_local std::unique_ptr<TaskPool> pool;
    if (pool && pool->owner != getpid()) {
        // in a forked child: the helpers stayed with the parent, so the
        // object is dropped without joining them
        (void)pool.release();
    }
    if (!pool) {
        const unsigned hw = std::thread::hardware_concurrency();
        pool.reset(new TaskPool((int)std::min<unsigned>(hw ? hw : 1, 32u) - 1));
    }
    return *pool;
}

// Host threads for the mesh and tree builds: f(task) for task in [0, ntask),
// handed out by an atomic counter to the calling thread and its pool of
// helpers (the hardware's thread count, at most 32, in all).  An exception
// from f is kept and rethrown, as a runtime_error, after all tasks ran.  f
// must not call parallel_tasks itself (the pool runs one job at a time).
template <class F>
void parallel_tasks(int64_t ntask, F &&f)
{
    if (ntask <= 0) return;
    if (ntask == 1) {
        f(0);
        return;
    }
    const std::function<void(int64_t)> fn = [&](int64_t t) { f(t); };
    thread_pool().run(ntask, fn);
}

// Touching triangles (sharing at least one vertex, itself included) of every
// triangle, with the shared-vertex count, as CSR in increasing triangle order.
// All phases on the host threads: the vertex -> triangle lists by atomic
// counts and cursors (their order is not kept: each triangle's list is
// sorted below), the triangles in chunks, and the chunks written into their
// final slots after a prefix sum of their sizes.
void build_adjacency(bem_mesh_s &M)
{
    const int64_t nt = M.nt, nv = M.nv;
    constexpr int64_t kChunk = 8192;
    const int64_t nchunk = (nt + kChunk - 1) / kChunk;
    std::vector<int64_t> vptr(nv + 1, 0);
    parallel_tasks(nchunk, [&](int64_t ck) {
        for (int64_t t = ck * kChunk, te = std::min(nt, t + kChunk); t < te; ++t)
            for (int a = 0; a < 3; ++a) __atomic_fetch_add(&vptr[M.T[3 * t + a] + 1], 1, __ATOMIC_RELAXED);
    });
    for (int64_t v = 0; v < nv; ++v) vptr[v + 1] += vptr[v];
    std::vector<int32_t, NoInit<int32_t>> vtri(vptr[nv]);
    std::vector<int64_t> fill(vptr.begin(), vptr.end() - 1);
    parallel_tasks(nchunk, [&](int64_t ck) {
        for (int64_t t = ck * kChunk, te = std::min(nt, t + kChunk); t < te; ++t)
            for (int a = 0; a < 3; ++a)
                vtri[__atomic_fetch_add(&fill[M.T[3 * t + a]], 1, __ATOMIC_RELAXED)] = (int32_t)t;
    });
    struct Part {
        std::vector<int64_t> len;
        std::vector<int32_t> tri;
        std::vector<int8_t> cs;
        int64_t max_touch = 0;
    };
    // each vertex's triangles in increasing order (the atomic fill leaves
    // them in any order)
    const int64_t nvchunk = (nv + kChunk - 1) / kChunk;
    parallel_tasks(nvchunk, [&](int64_t ck) {
        for (int64_t v = ck * kChunk, ve = std::min(nv, v + kChunk); v < ve; ++v)
            std::sort(vtri.begin() + vptr[v], vtri.begin() + vptr[v + 1]);
    });
    // the triangles touching t: a three-way merge of its vertices' sorted
    // lists, each triangle once, with the number of lists that hold it (the
    // vertices it shares with t: 1 vertex, 2 edge, 3 t itself)
    std::vector<Part> parts(nchunk);
    parallel_tasks(nchunk, [&](int64_t ck) {
        Part P;  // moved in at the end: neighbouring chunks' parts share cache lines
        const int64_t t0 = ck * kChunk, t1 = std::min(nt, t0 + kChunk);
        P.len.reserve(t1 - t0);
        P.tri.reserve(16 * (t1 - t0));
        P.cs.reserve(16 * (t1 - t0));
        for (int64_t t = t0; t < t1; ++t) {
            const int32_t *l[3], *le[3];
            for (int a = 0; a < 3; ++a) {
                const int32_t v = M.T[3 * t + a];
                l[a] = vtri.data() + vptr[v];
                le[a] = vtri.data() + vptr[v + 1];
            }
            int64_t cnt = 0;
            for (;;) {
                int32_t m = INT32_MAX;
                bool any = false;
                for (int a = 0; a < 3; ++a)
                    if (l[a] < le[a] && (!any || *l[a] < m)) {
                        m = *l[a];
                        any = true;
                    }
                if (!any) break;
                int8_t k = 0;
                for (int a = 0; a < 3; ++a)
                    if (l[a] < le[a] && *l[a] == m) {
                        ++l[a];
                        ++k;
                    }
                P.tri.push_back(m);
                P.cs.push_back(k);
                ++cnt;
            }
            P.len.push_back(cnt);
            P.max_touch = std::max(P.max_touch, cnt);
        }
        parts[ck] = std::move(P);
    });
    std::vector<int64_t> off(nchunk + 1, 0);
    M.max_touch = 0;
    for (int64_t ck = 0; ck < nchunk; ++ck) {
        off[ck + 1] = off[ck] + (int64_t)parts[ck].tri.size();
        M.max_touch = std::max(M.max_touch, parts[ck].max_touch);
    }
    M.adj_ptr.resize(nt + 1);
    M.adj_tri.resize(off[nchunk]);
    M.adj_case.resize(off[nchunk]);
    parallel_tasks(nchunk, [&](int64_t ck) {
        const Part &P = parts[ck];
        std::copy(P.tri.begin(), P.tri.end(), M.adj_tri.begin() + off[ck]);
        std::copy(P.cs.begin(), P.cs.end(), M.adj_case.begin() + off[ck]);
        int64_t o = off[ck];
        for (size_t q = 0; q < P.len.size(); ++q) {
            M.adj_ptr[ck * kChunk + (int64_t)q] = o;
            o += P.len[q];
        }
    });
    M.adj_ptr[nt] = off[nchunk];
}

}  // namespace

namespace bem {

bool mesh_view(const void *mesh, MeshView *out)
{
    if (!mesh || !out) return false;
    const bem_mesh_s *M = static_cast<const bem_mesh_s *>(mesh);
    out->g = M->geom.g;
    out->device = M->device;
    out->nt = M->nt;
    out->max_touch = M->max_touch;
    return true;
}

bool consts_peek(int device, QuadRule *rule, const SingTable **sing)
{
    std::lock_guard<std::mutex> lk(g_dev_mu);
    auto it = g_dev.find(device);
    if (it == g_dev.end()) return false;
    *rule = it->second->rule;
    *sing = it->second->sing;
    return true;
}

void set_last_error(const char *msg) { g_err = msg ? msg : ""; }

}  // namespace bem

extern "C" {

int bem_version(void) { return 100; }

int64_t bem_kernel_launches(void) { return launches_total(); }

int bem_memory_usage(int64_t *reserved, int64_t *used)
{
    return guarded([&]() -> int {
        cudaMemPool_t pool = lib_pool();
        uint64_t r = 0, u = 0;
        CU(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r));
        CU(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u));
        if (reserved) *reserved = (int64_t)r;
        if (used) *used = (int64_t)u;
        return BEM_OK;
    });
}

int bem_debug_recip(const double *x, double *y, int64_t n, void *cuda_stream)
{
    return guarded([&]() -> int {
        if (n < 0) return fail(BEM_E_ARG, "negative size");
        if (n == 0) return BEM_OK;
        if (!x || !y) return fail(BEM_E_ARG, "null array");
        cudaStream_t st = (cudaStream_t)cuda_stream;
        CU(launch_debug_recip(x, y, n, st));
        CU(cudaStreamSynchronize(st));
        return BEM_OK;
    });
}

int bem_debug_rsqrt(const double *x, double *y, int64_t n, void *cuda_stream)
{
    return guarded([&]() -> int {
        if (n < 0) return fail(BEM_E_ARG, "negative size");
        if (n == 0) return BEM_OK;
        if (!x || !y) return fail(BEM_E_ARG, "null array");
        cudaStream_t st = (cudaStream_t)cuda_stream;
        CU(launch_debug_rsqrt(x, y, n, st));
        CU(cudaStreamSynchronize(st));
        return BEM_OK;
    });
}

int bem_set_tuning(const bem_tuning *t)
{
    if (!t || t->warp_max_rows < 1 || t->warp_max_rows > aca_small_cap() || t->lane_max_rows < 0 ||
        t->lane_max_rows > aca_tiny_max() || t->lane_max_rows > t->warp_max_rows ||
        (t->use_graphs != 0 && t->use_graphs != 1)) {
        set_last_error("bad tuning values");
        return BEM_E_ARG;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuning = *t;
    return BEM_OK;
}

int bem_get_tuning(bem_tuning *t)
{
    if (!t) return BEM_E_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    *t = g_tuning;
    return BEM_OK;
}

int bem_set_quadrature(const bem_quadrature *q)
{
    if (!q || !(q->rho3 >= 0.0) || !(q->rho1 >= 0.0) || !std::isfinite(q->rho3) ||
        !std::isfinite(q->rho1))
        return fail(BEM_E_ARG, "quadrature thresholds must be finite and >= 0");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_quad = *q;
    return BEM_OK;
}

int bem_get_quadrature(bem_quadrature *q)
{
    if (!q) return BEM_E_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    *q = g_quad;
    return BEM_OK;
}

const char *bem_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace bem {

int mesh_upload(bem_mesh M, cudaStream_t st);

// Mesh creation with all device work on stream st (synchronised before return);
// st == kHostOnly stops after the host part (validation and adjacency).
int mesh_create_impl(const double *vertices, int64_t n_vertices, const int32_t *triangles,
                     int64_t n_triangles, cudaStream_t st, bem_mesh *out)
{
    return guarded([&]() -> int {
        if (!out) return fail(BEM_E_ARG, "out is null");
        *out = nullptr;
        if (!vertices || !triangles) return fail(BEM_E_ARG, "null input array");
        if (n_vertices < 3 || n_triangles < 1 || n_triangles >= (int64_t(1) << 31) ||
            n_vertices >= (int64_t(1) << 31))
            return fail(BEM_E_ARG, "bad mesh sizes");
        auto M = std::make_unique<bem_mesh_s>();
        M->nv = n_vertices;
        M->nt = n_triangles;
        M->V.assign(vertices, vertices + 3 * n_vertices);
        M->T.assign(triangles, triangles + 3 * n_triangles);
        // validation in chunks on the host threads; each chunk keeps its first
        // failure, and the smallest index over the chunks is reported (the
        // one a sequential scan finds first)
        constexpr int64_t kVal = 65536;
        const int64_t nvc = (3 * n_vertices + kVal - 1) / kVal;
        std::vector<int64_t> bad_v(nvc, -1);
        parallel_tasks(nvc, [&](int64_t ck) {
            for (int64_t i = ck * kVal, ie = std::min(3 * n_vertices, i + kVal); i < ie; ++i)
                if (!std::isfinite(M->V[i])) {
                    bad_v[ck] = i;
                    return;
                }
        });
        for (int64_t i : bad_v)
            if (i >= 0)
                return fail(BEM_E_MESH, "non-finite coordinate at vertex " + std::to_string(i / 3));
        const int64_t ntc = (n_triangles + kVal - 1) / kVal;
        std::vector<int64_t> bad_t(ntc, -1);
        std::vector<int> bad_kind(ntc, 0);
        parallel_tasks(ntc, [&](int64_t ck) {
            for (int64_t t = ck * kVal, te = std::min(n_triangles, t + kVal); t < te; ++t) {
                const int32_t *tr = &M->T[3 * t];
                int kind = 0;
                for (int a = 0; a < 3; ++a)
                    if (tr[a] < 0 || tr[a] >= n_vertices) kind = 1;
                if (!kind && (tr[0] == tr[1] || tr[1] == tr[2] || tr[0] == tr[2])) kind = 2;
                if (!kind) {
                    const double *a = &M->V[3 * tr[0]], *b = &M->V[3 * tr[1]], *c = &M->V[3 * tr[2]];
                    double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
                    double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
                    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                                   e1[0] * e2[1] - e1[1] * e2[0]};
                    double n2 = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
                    double s2 = (e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]) *
                                (e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]);
                    if (!(n2 > 1e-24 * s2) || n2 == 0.0) kind = 3;
                }
                if (kind) {
                    bad_t[ck] = t;
                    bad_kind[ck] = kind;
                    return;
                }
            }
        });
        for (int64_t ck = 0; ck < ntc; ++ck) {
            if (bad_t[ck] < 0) continue;
            const std::string ts = std::to_string(bad_t[ck]);
            if (bad_kind[ck] == 1) return fail(BEM_E_MESH, "vertex index out of range in triangle " + ts);
            if (bad_kind[ck] == 2) return fail(BEM_E_MESH, "repeated vertex in triangle " + ts);
            return fail(BEM_E_MESH, "zero-area triangle " + ts);
        }
        build_adjacency(*M);
        if (st != kHostOnly) {
            int rc = mesh_upload(M.get(), st);
            if (rc) return rc;
        }
        *out = M.release();
        return BEM_OK;
    });
}

// Device part of a mesh: geometry on stream st (synchronised).
int mesh_upload(bem_mesh M, cudaStream_t st)
{
    return guarded([&]() -> int {
        CU(cudaGetDevice(&M->device));
        DeviceConsts &D = device_consts();
        M->dV.upload(M->V, st);
        M->dT.upload(M->T, st);
        M->geom.build(M->dV.as<double>(), M->dT.as<int32_t>(), nullptr, M->nt, D.rule, st);
        CU(cudaStreamSynchronize(st));
        return BEM_OK;
    });
}

// Frees a mesh whose streams have all been synchronised by the caller.
void mesh_free_synced(bem_mesh M) { delete M; }

}  // namespace bem

extern "C" {

int bem_mesh_create(const double *vertices, int64_t n_vertices, const int32_t *triangles,
                    int64_t n_triangles, bem_mesh *out)
{
    return mesh_create_impl(vertices, n_vertices, triangles, n_triangles, 0, out);
}

int bem_mesh_destroy(bem_mesh mesh)
{
    return guarded([&]() -> int {
        if (!mesh) return fail(BEM_E_ARG, "null mesh");
        if (mesh->hmat_refs > 0) return fail(BEM_E_STATE, "H-matrices still use this mesh");
        cudaDeviceSynchronize();  // work of any stream may still read the mesh
        delete mesh;
        return BEM_OK;
    });
}

int64_t bem_mesh_size(bem_mesh mesh) { return mesh ? mesh->nt : -1; }

int bem_entries(bem_mesh mesh, int32_t op, double k, int32_t prec, const int32_t *test_ids,
                int64_t n_test, const int32_t *trial_ids, int64_t n_trial, void *out,
                void *cuda_stream)
{
    return guarded([&]() -> int {
        if (!mesh) return fail(BEM_E_ARG, "null mesh");
        if (op < 0 || op > 2) return fail(BEM_E_ARG, "bad op");
        if (prec != BEM_FP64 && prec != BEM_MIXED && prec != BEM_MIXED_SP) return fail(BEM_E_ARG, "bad prec");
        if (!std::isfinite(k)) return fail(BEM_E_ARG, "bad k");
        if (n_test < 0 || n_trial < 0) return fail(BEM_E_ARG, "negative size");
        if (n_test == 0 || n_trial == 0) return BEM_OK;
        if (!test_ids || !trial_ids || !out) return fail(BEM_E_ARG, "null array");
        cudaStream_t st = (cudaStream_t)cuda_stream;
        DeviceConsts &D = device_consts();
        const bool cplx = k != 0.0;
        const size_t esz = cplx ? 16 : 8;
        const int64_t nout = n_test * n_trial;
        // stage host arrays
        DBuf sti, stj, sto;
        const int32_t *dti = test_ids, *dtj = trial_ids;
        void *dout = out;
        bool host_out = !is_device_ptr(out);
        if (!is_device_ptr(test_ids)) {
            for (int64_t a = 0; a < n_test; ++a)
                if (test_ids[a] < 0 || test_ids[a] >= mesh->nt)
                    return fail(BEM_E_ARG, "test id out of range");
            sti.alloc(n_test * 4, st);
            CU(cudaMemcpyAsync(sti.p, test_ids, n_test * 4, cudaMemcpyHostToDevice, st));
            dti = sti.as<int32_t>();
        }
        if (!is_device_ptr(trial_ids)) {
            for (int64_t b = 0; b < n_trial; ++b)
                if (trial_ids[b] < 0 || trial_ids[b] >= mesh->nt)
                    return fail(BEM_E_ARG, "trial id out of range");
            stj.alloc(n_trial * 4, st);
            CU(cudaMemcpyAsync(stj.p, trial_ids, n_trial * 4, cudaMemcpyHostToDevice, st));
            dtj = stj.as<int32_t>();
        }
        if (host_out) {
            sto.alloc(nout * esz, st);
            dout = sto.p;
        }
        // scratch: singular pair lists (one per case), counters, error flag.
        // The bound counts n_test * (most triangles touching one triangle);
        // repeated trial ids can exceed it, and then the counters (which keep
        // counting past the capacity) size a second pass
        unsigned long long cap =
            (unsigned long long)std::min<int64_t>(nout, n_test * std::max<int64_t>(mesh->max_touch, 1));
        int herr = 0;
        for (int pass = 0; pass < 2; ++pass) {
            size_t list_bytes = cap * sizeof(SingPair);
            size_t scratch = 3 * list_bytes + 64;
            void *ws = nullptr;
            CU(lib_malloc_async(&ws, scratch, st));
            unsigned char *wb = (unsigned char *)ws;
            SingPair *lists[3] = {(SingPair *)wb, (SingPair *)(wb + list_bytes),
                                  (SingPair *)(wb + 2 * list_bytes)};
            unsigned long long *counts = (unsigned long long *)(wb + 3 * list_bytes);
            int *err = (int *)(counts + 3);
            unsigned long long hcount[3] = {0, 0, 0};
            cudaError_t e = cudaMemsetAsync(counts, 0, 64, st);
            if (e == cudaSuccess)
                e = launch_entries_regular(mesh->geom.g, D.rule, op, k, prec, dti, n_test, dtj,
                                           n_trial, dout, lists, counts, cap, err, st);
            const SingPair *cl[3] = {lists[0], lists[1], lists[2]};
            int64_t hc[3] = {(int64_t)cap, (int64_t)cap, (int64_t)cap};
            if (e == cudaSuccess) e = launch_singular(mesh->geom.g, D.sing, op, k, prec, cl, counts, hc, dout, st);
            herr = 0;
            if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(hcount, counts, sizeof(hcount), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            cudaFreeAsync(ws, st);
            if (e != cudaSuccess) {
                g_err = std::string("bem_entries: ") + cudaGetErrorString(e);
                return e == cudaErrorMemoryAllocation ? BEM_E_OOM : BEM_E_CUDA;
            }
            if (herr != 2) break;
            cap = std::max({hcount[0], hcount[1], hcount[2]});
        }
        if (herr == 0 && host_out) {
            CU(cudaMemcpyAsync(out, dout, nout * esz, cudaMemcpyDeviceToHost, st));
            CU(cudaStreamSynchronize(st));
        }
        if (herr == 1) return fail(BEM_E_ARG, "triangle id out of range");
        if (herr == 2) return fail(BEM_E_CUDA, "singular pair list overflow");
        return BEM_OK;
    });
}

int bem_entries_dp1(bem_mesh mesh, int32_t op, double k, int32_t prec, const int32_t *test_tris,
                    int64_t n_test, const int32_t *trial_tris, int64_t n_trial, void *out,
                    void *cuda_stream)
{
    return guarded([&]() -> int {
        if (!mesh) return fail(BEM_E_ARG, "null mesh");
        if (op < 0 || op > 2) return fail(BEM_E_ARG, "bad op");
        if (prec != BEM_FP64 && prec != BEM_MIXED) return fail(BEM_E_ARG, "bad prec");
        if (!std::isfinite(k)) return fail(BEM_E_ARG, "bad k");
        if (n_test < 0 || n_trial < 0) return fail(BEM_E_ARG, "negative size");
        if (n_test == 0 || n_trial == 0) return BEM_OK;
        if (3 * n_trial >= (int64_t(1) << 31)) return fail(BEM_E_ARG, "n_trial too large");
        if (!test_tris || !trial_tris || !out) return fail(BEM_E_ARG, "null array");
        cudaStream_t st = (cudaStream_t)cuda_stream;
        DeviceConsts &D = device_consts();
        const bool cplx = k != 0.0;
        const size_t esz = cplx ? 16 : 8;
        const int64_t nout = 9 * n_test * n_trial;
        DBuf sti, stj, sto;
        const int32_t *dti = test_tris, *dtj = trial_tris;
        void *dout = out;
        const bool host_out = !is_device_ptr(out);
        if (!is_device_ptr(test_tris)) {
            for (int64_t a = 0; a < n_test; ++a)
                if (test_tris[a] < 0 || test_tris[a] >= mesh->nt)
                    return fail(BEM_E_ARG, "test id out of range");
            sti.alloc(n_test * 4, st);
            CU(cudaMemcpyAsync(sti.p, test_tris, n_test * 4, cudaMemcpyHostToDevice, st));
            dti = sti.as<int32_t>();
        }
        if (!is_device_ptr(trial_tris)) {
            for (int64_t b = 0; b < n_trial; ++b)
                if (trial_tris[b] < 0 || trial_tris[b] >= mesh->nt)
                    return fail(BEM_E_ARG, "trial id out of range");
            stj.alloc(n_trial * 4, st);
            CU(cudaMemcpyAsync(stj.p, trial_tris, n_trial * 4, cudaMemcpyHostToDevice, st));
            dtj = stj.as<int32_t>();
        }
        if (host_out) {
            sto.alloc(nout * esz, st);
            dout = sto.p;
        }
        // scratch: touching-pair lists (one per case), counters, error flag
        const unsigned long long cap = (unsigned long long)std::min<int64_t>(
            n_test * n_trial, n_test * std::max<int64_t>(mesh->max_touch, 1));
        const size_t list_bytes = cap * sizeof(SingPairL);
        void *ws = nullptr;
        CU(lib_malloc_async(&ws, 3 * list_bytes + 64, st));
        unsigned char *wb = (unsigned char *)ws;
        SingPairL *lists[3] = {(SingPairL *)wb, (SingPairL *)(wb + list_bytes),
                               (SingPairL *)(wb + 2 * list_bytes)};
        unsigned long long *counts = (unsigned long long *)(wb + 3 * list_bytes);
        int *err = (int *)(counts + 3);
        cudaError_t e = cudaMemsetAsync(counts, 0, 64, st);
        if (e == cudaSuccess)
            e = launch_entries_dp1(mesh->geom.g, D.rule, op, k, prec, dti, n_test, dtj, n_trial,
                                   dout, lists, counts, cap, err, st);
        const SingPairL *cl[3] = {lists[0], lists[1], lists[2]};
        const int64_t hc[3] = {(int64_t)cap, (int64_t)cap, (int64_t)cap};
        if (e == cudaSuccess)
            e = launch_singular_dp1(mesh->geom.g, D.sing, op, k, cl, counts, hc, dout, st);
        int herr = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && host_out)
            e = cudaMemcpyAsync(out, dout, nout * esz, cudaMemcpyDeviceToHost, st);
        cudaFreeAsync(ws, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            g_err = std::string("bem_entries_dp1: ") + cudaGetErrorString(e);
            return e == cudaErrorMemoryAllocation ? BEM_E_OOM : BEM_E_CUDA;
        }
        if (herr == 1) return fail(BEM_E_ARG, "triangle id out of range");
        if (herr == 2) return fail(BEM_E_CUDA, "singular pair list overflow");
        return BEM_OK;
    });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// H-matrices
// ---------------------------------------------------------------------------
struct Cluster {
    int64_t b, e, left, right;
    double box[6];
    double h = 0.0;  // longest edge of any of its triangles
};

struct BlockH {
    int64_t tau, sigma;
    bool adm;
};

struct bem_hmat_s {
    bem_mesh mesh = nullptr;
    int leaf = 0;
    double eta = 0;
    // function space: BEM_P0 (a dof per triangle) or the piecewise linear
    // spaces, held as DP1 (three local dofs per triangle: dof 3 t + a is the
    // local basis function of vertex a of triangle t); BEM_P1 applies the
    // continuous space's transforms around the DP1 matrix in products
    int space = BEM_P0;
    int dofs = 1;
    int64_t ndof = 0;                     // length of the internal vectors
    int64_t row_b = 0, row_e = -1;        // cluster-order rows kept (a part of a row partition)
    std::vector<int32_t> dperm;           // dof permutation (DP1): cluster dof -> mesh dof
    std::vector<SingPairL, NoInit<SingPairL>> singl[3];  // touching pairs of the DP1 near field
    std::vector<int64_t> vptr;            // P1: per vertex, its DP1 dofs (CSR, mesh order)
    std::vector<int32_t> vdof;
    double rho3 = 0.0, rho1 = 0.0;        // distance-class thresholds of the regular rules
    bool has_rules = false;               // some admissible block uses a lower-order rule
    int64_t small_max = 8192;             // blocks with max(m, n) <= this run on one warp
    int64_t tiny_max = 0;                 // ... and with max(m, n) <= this on one lane
    std::vector<int32_t> perm, iperm;
    std::vector<Cluster> cl;
    std::vector<BlockH> blocks;           // tree order
    std::vector<NearBlock, NoInit<NearBlock>> near;     // host copies
    std::vector<int64_t, NoInit<int64_t>> near_block_id;  // index into blocks
    std::vector<FarBlock, NoInit<FarBlock>> far;  // LPT order (big first, then small)
    std::vector<int64_t, NoInit<int64_t>> far_block_id;
    int64_t nshape[5] = {0, 0, 0, 0, 0};  // admissible blocks per work shape (AcaShape)
    int64_t max_m_big = 0, max_m_small = 0;
    int64_t near_total = 0;
    std::vector<SingPair, NoInit<SingPair>> sing[3];
    // per vertex-adjacent pair of sing[0] (P0): the offset of the transposed
    // entry, evaluated by the same quadrature, or -1
    std::vector<int64_t, NoInit<int64_t>> sing_t;
    int64_t sing_entries[3] = {0, 0, 0};  // entries the pair lists write
    // leaves (matvec)
    std::vector<int64_t> leaf_rows, leaf_ptr;
    std::vector<int64_t, NoInit<int64_t>> leaf_items;
    // device
    DBuf d_perm, d_near, d_far, d_chunks, d_sing[3], d_sing_t, d_leaf_rows, d_leaf_ptr, d_leaf_items, d_long, d_long_off;
    std::vector<int64_t> long_ids;        // admissible blocks with long columns (matvec)
    DBuf d_near_data, d_pool, d_poolhdr, d_queue, d_toff, d_xt, d_yt, d_tbuf, d_x, d_y;
    DBuf d_dperm, d_singl[3], d_vptr, d_vdof, d_xs, d_ys;
    GeomStore geom;                       // cluster order
    // assembled state
    bool assembled = false;
    int op = 0, prec = 0;
    double k = 0.0, eps = 0.0;
    bool cplx = false;
    std::vector<int64_t> toff;
    std::vector<FarBlock> far_result;     // host copy of the factor descriptors, fetched lazily
    bool far_result_valid = false;
    int64_t factor_elems = 0, k2mn = 0, rank_mn = 0;
    DBuf d_tiles, d_acastats, d_job;
    int64_t pool_elems = 0, pool_want = 0;
    double t_tree = 0, t_near = 0, t_far = 0, t_near_reg = 0;
    double t_clusters = 0, t_blocks = 0, t_lists = 0, t_upload = 0;
    // CUDA graph of the assembly sequence and what it was captured for
    cudaGraphExec_t graph = nullptr;
    int g_op = -1, g_prec = -1;
    double g_k = 0, g_eps = 0;
    void *g_pool = nullptr, *g_near = nullptr;
    int64_t g_nodes = 0, g_pool_elems = -1;
    // timing: 0 start, 1 end of the near field, 2 end of the ACA, 3 end of the
    // regular near pairs, 4 start of the ACA
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaStream_t cap_stream = nullptr;
    Pool *pin_pool = nullptr;       // pinned readback slots
    AcaStats *pin_stats = nullptr;
    AcaJob *pin_job = nullptr;      // pinned source of d_job (this matrix as one ACA job)
    ~bem_hmat_s()
    {
        pinned_release(pin_job);
        if (graph) cudaGraphExecDestroy(graph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        pinned_release(pin_pool);
        pinned_release(pin_stats);
    }
    int64_t far_entries = 0, rank_sum = 0, capped = 0;
    int32_t rank_min = 0, rank_max = 0;
};

namespace {

// Cluster tree (Sec. 2.1): a cluster with more than leaf_size triangles is
// split along the longest axis of its vertex bounding box at the median of
// the centroids ((v0 + v1) + v2) / 3, ties by triangle index; leaves list
// their triangles in increasing index order.  Breadth-first numbering.
// One cluster: its vertex box, and either its leaf order or its split (the
// median of the centroids along the longest box axis).  Returns the split
// point, or -1 for a leaf.
int64_t split_cluster(Cluster &C, std::vector<int32_t> &perm,
                      const std::vector<double, NoInit<double>> &cen,
                      const std::vector<double, NoInit<double>> &tbox,
                      const std::vector<double, NoInit<double>> &tlen, int leaf)
{
    double box[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    double h = 0.0;
    for (int64_t q = C.b; q < C.e; ++q) {
        const double *tb = &tbox[6 * (int64_t)perm[q]];
        for (int c = 0; c < 3; ++c) {
            box[c] = std::min(box[c], tb[c]);
            box[3 + c] = std::max(box[3 + c], tb[3 + c]);
        }
        h = std::max(h, tlen[perm[q]]);
    }
    std::memcpy(C.box, box, sizeof(box));
    C.h = h;
    const int64_t n = C.e - C.b;
    if (n <= leaf) {
        std::sort(perm.begin() + C.b, perm.begin() + C.e);
        return -1;
    }
    int axis = 0;
    double ext = box[3] - box[0];
    for (int a = 1; a < 3; ++a)
        if (box[3 + a] - box[a] > ext) {
            ext = box[3 + a] - box[a];
            axis = a;
        }
    auto less = [&](int32_t x, int32_t y) {
        double cx = cen[3 * (int64_t)x + axis], cy = cen[3 * (int64_t)y + axis];
        return cx < cy || (cx == cy && x < y);
    };
    const int64_t mid = C.b + n / 2;
    std::nth_element(perm.begin() + C.b, perm.begin() + mid, perm.begin() + C.e, less);
    return mid;
}

// Sub-phase timings of the tree build on stderr when BEM_TRACE_TREE is set.
struct PhaseTrace {
    bool on;
    const char *label;
    double t0, last;
    std::string text;
    explicit PhaseTrace(const char *what)
        : on(std::getenv("BEM_TRACE_TREE") != nullptr), label(what), t0(now_ms()), last(t0)
    {
    }
    void mark(const char *name)
    {
        if (!on) return;
        const double t = now_ms();
        char buf[96];
        std::snprintf(buf, sizeof buf, " %s %.2f", name, t - last);
        text += buf;
        last = t;
    }
    ~PhaseTrace()
    {
        if (on) std::fprintf(stderr, "tree %s (ms):%s; total %.2f\n", label, text.c_str(), now_ms() - t0);
    }
};

// The tree is grown breadth-first until there are enough clusters to keep
// the host threads busy; the subtrees below that frontier are grown on the
// threads (each in its own list, depth-first) and appended in frontier order.
// The splits, and so the partition, the block tree and every block list, are
// those of the sequential breadth-first construction; only the cluster
// numbering below the frontier differs.
void build_clusters(bem_hmat_s &H)
{
    PhaseTrace trace("clusters");
    const bem_mesh_s &M = *H.mesh;
    const int64_t nt = M.nt;
    std::vector<double, NoInit<double>> cen(3 * nt), tbox(6 * nt), tlen(nt);
    parallel_tasks((nt + 16383) / 16384, [&](int64_t task) {
        for (int64_t t = task * 16384, te = std::min(nt, t + 16384); t < te; ++t) {
            // longest edge (squared lengths compared, one square root)
            double h2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                const double *u = &M.V[3 * (int64_t)M.T[3 * t + a]];
                const double *v = &M.V[3 * (int64_t)M.T[3 * t + (a + 1) % 3]];
                double l2 = 0.0;
                for (int c = 0; c < 3; ++c) l2 += (u[c] - v[c]) * (u[c] - v[c]);
                h2 = std::max(h2, l2);
            }
            tlen[t] = std::sqrt(h2);
            for (int c = 0; c < 3; ++c) {
                const double a = M.V[3 * (int64_t)M.T[3 * t] + c], b = M.V[3 * (int64_t)M.T[3 * t + 1] + c],
                             d = M.V[3 * (int64_t)M.T[3 * t + 2] + c];
                cen[3 * t + c] = ((a + b) + d) / 3.0;
                tbox[6 * t + c] = std::min(std::min(a, b), d);
                tbox[6 * t + 3 + c] = std::max(std::max(a, b), d);
            }
        }
    });
    trace.mark("triangles");
    H.perm.resize(nt);
    std::iota(H.perm.begin(), H.perm.end(), 0);
    H.cl.clear();
    H.cl.push_back({0, nt, -1, -1, {0, 0, 0, 0, 0, 0}});
    unsigned hw = std::thread::hardware_concurrency();
    const size_t want = 2 * (size_t)std::max(1u, std::min(hw, 32u));
    // breadth-first top: the clusters of [head, size) are the frontier
    size_t head = 0;
    while (head < H.cl.size() && H.cl.size() - head < want) {
        const size_t end = H.cl.size();
        // the clusters of one level own disjoint ranges of perm: split them
        // on the threads, then append their children in order
        std::vector<int64_t> mids(end - head);
        parallel_tasks((int64_t)(end - head), [&](int64_t i) {
            Cluster C = H.cl[head + i];
            mids[i] = split_cluster(C, H.perm, cen, tbox, tlen, H.leaf);
            H.cl[head + i] = C;
        });
        for (size_t q = head; q < end; ++q) {
            const Cluster C = H.cl[q];
            const int64_t mid = mids[q - head];
            if (mid >= 0) {
                const int64_t L = (int64_t)H.cl.size();
                H.cl[q].left = L;
                H.cl[q].right = L + 1;
                H.cl.push_back({C.b, mid, -1, -1, {0, 0, 0, 0, 0, 0}});
                H.cl.push_back({mid, C.e, -1, -1, {0, 0, 0, 0, 0, 0}});
            }
        }
        head = end;
        bool any_split = false;
        for (size_t q = head; q < H.cl.size(); ++q) any_split |= H.cl[q].e - H.cl[q].b > H.leaf;
        if (!any_split) break;
    }
    trace.mark("top_levels");
    // subtrees of the frontier clusters, one task each (disjoint perm ranges)
    const size_t nfront = H.cl.size() - head;
    std::vector<std::vector<Cluster>> sub(nfront);
    parallel_tasks((int64_t)nfront, [&](int64_t f) {
        std::vector<Cluster> S;  // moved in at the end (neighbouring headers share cache lines)
        S.push_back(H.cl[head + f]);
        for (size_t q = 0; q < S.size(); ++q) {
            Cluster C = S[q];
            const int64_t mid = split_cluster(C, H.perm, cen, tbox, tlen, H.leaf);
            if (mid >= 0) {
                C.left = (int64_t)S.size();   // local index, fixed up below
                C.right = C.left + 1;
                S[q] = C;
                S.push_back({C.b, mid, -1, -1, {0, 0, 0, 0, 0, 0}});
                S.push_back({mid, C.e, -1, -1, {0, 0, 0, 0, 0, 0}});
            } else {
                S[q] = C;
            }
        }
        sub[f] = std::move(S);
    });
    trace.mark("subtrees");
    // the frontier cluster keeps its index; its descendants follow in order
    for (size_t f = 0; f < nfront; ++f) {
        const int64_t base = (int64_t)H.cl.size() - 1;   // local index 1 -> base + 1
        const std::vector<Cluster> &S = sub[f];
        auto fix = [&](int64_t l) { return l < 0 ? l : base + l; };
        Cluster root = S[0];
        root.left = fix(root.left);
        root.right = fix(root.right);
        H.cl[head + f] = root;
        for (size_t q = 1; q < S.size(); ++q) {
            Cluster C = S[q];
            C.left = fix(C.left);
            C.right = fix(C.right);
            H.cl.push_back(C);
        }
    }
    trace.mark("join");
    H.iperm.resize(nt);
    parallel_tasks((nt + 65535) / 65536, [&](int64_t task) {
        for (int64_t p = task * 65536, pe = std::min(nt, p + 65536); p < pe; ++p)
            H.iperm[H.perm[p]] = (int32_t)p;
    });
}

// Admissibility (Sec. 2.1): disjoint boxes and min(diam) <= eta * dist.
bool admissible(const double *bt, const double *bs, double eta)
{
    double dt = std::sqrt((bt[3] - bt[0]) * (bt[3] - bt[0]) + (bt[4] - bt[1]) * (bt[4] - bt[1]) +
                          (bt[5] - bt[2]) * (bt[5] - bt[2]));
    double ds = std::sqrt((bs[3] - bs[0]) * (bs[3] - bs[0]) + (bs[4] - bs[1]) * (bs[4] - bs[1]) +
                          (bs[5] - bs[2]) * (bs[5] - bs[2]));
    double g[3];
    for (int c = 0; c < 3; ++c) {
        double g1 = bs[c] - bt[3 + c], g2 = bt[c] - bs[3 + c];
        double m = g1 > g2 ? g1 : g2;
        g[c] = m > 0 ? m : 0;
    }
    double dist = std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (!(dist > 0)) return false;
    return (dt < ds ? dt : ds) <= eta * dist;
}

// Regular rule of an admissible block by its distance class: rho = dist / h,
// dist the distance between the cluster boxes (as in the admissibility test)
// and h the longest triangle edge in either cluster; rho >= rho1 > 0 gives
// the centroid rule, else rho >= rho3 > 0 the 3-point degree-2 rule, else the
// 6-point degree-4 rule of Sec. 3.2.1.
int block_rule(const Cluster &T, const Cluster &S, double rho3, double rho1)
{
    if (!(rho3 > 0) && !(rho1 > 0)) return kRule6;
    const double *bt = T.box, *bs = S.box;
    double g2 = 0.0;
    for (int c = 0; c < 3; ++c) {
        const double g1 = bs[c] - bt[3 + c], gb = bt[c] - bs[3 + c];
        const double m = g1 > gb ? g1 : gb;
        if (m > 0) g2 += m * m;
    }
    const double dist = std::sqrt(g2), h = std::max(T.h, S.h);
    if (rho1 > 0 && dist >= rho1 * h) return kRule1;
    if (rho3 > 0 && dist >= rho3 * h) return kRule3;
    return kRule6;
}

// Block tree: pairs (tau, sigma) from (root, root); an admissible pair, or one
// with a leaf, is a block; otherwise its children pairs are visited in the
// order (l,l), (l,r), (r,l), (r,r).  The blocks are listed depth-first ("tree
// order").  The top of the tree is expanded level by level, which keeps that
// order, until there are enough pairs for the host threads; the subtrees of
// the remaining pairs are expanded depth-first on the threads and their
// blocks concatenated in order.
void build_blocks(bem_hmat_s &H)
{
    H.blocks.clear();
    struct Item {
        int64_t t, s;
        int8_t state;  // 0 open, 1 admissible block, 2 dense block
    };
    auto classify = [&](int64_t t, int64_t s) -> int8_t {
        const Cluster &T = H.cl[t], &S = H.cl[s];
        const bool adm = admissible(T.box, S.box, H.eta);
        if (adm) return 1;
        if (T.left < 0 || S.left < 0) return 2;
        return 0;
    };
    unsigned hw = std::thread::hardware_concurrency();
    const size_t want = 8 * (size_t)std::max(1u, std::min(hw, 32u));
    std::vector<Item> front{{0, 0, classify(0, 0)}};
    for (;;) {
        size_t open = 0;
        for (const Item &it : front) open += it.state == 0;
        if (open == 0 || open >= want) break;
        std::vector<Item> next;
        next.reserve(front.size() + 3 * open);
        for (const Item &it : front) {
            if (it.state != 0) {
                next.push_back(it);
                continue;
            }
            const Cluster &T = H.cl[it.t], &S = H.cl[it.s];
            const int64_t ch[4][2] = {{T.left, S.left}, {T.left, S.right}, {T.right, S.left},
                                      {T.right, S.right}};
            for (auto &c : ch) next.push_back({c[0], c[1], classify(c[0], c[1])});
        }
        front.swap(next);
    }
    std::vector<std::vector<BlockH>> sub(front.size());
    parallel_tasks((int64_t)front.size(), [&](int64_t f) {
        const Item &it = front[f];
        std::vector<BlockH> out;  // moved in at the end (neighbouring headers share cache lines)
        if (it.state != 0) {
            out.push_back({it.t, it.s, it.state == 1});
            sub[f] = std::move(out);
            return;
        }
        std::vector<std::pair<int64_t, int64_t>> stack{{it.t, it.s}};
        while (!stack.empty()) {
            auto [t, s] = stack.back();
            stack.pop_back();
            const int8_t st = classify(t, s);
            if (st != 0) {
                out.push_back({t, s, st == 1});
                continue;
            }
            const Cluster &T = H.cl[t], &S = H.cl[s];
            stack.push_back({T.right, S.right});
            stack.push_back({T.right, S.left});
            stack.push_back({T.left, S.right});
            stack.push_back({T.left, S.left});
        }
        sub[f] = std::move(out);
    });
    size_t total = 0;
    for (auto &v : sub) total += v.size();
    H.blocks.reserve(total);
    for (auto &v : sub) H.blocks.insert(H.blocks.end(), v.begin(), v.end());
}

// Block lists.  Near-field blocks keep tree order and get consecutive dense
// storage.  Admissible blocks are split into classes by their longer side
// (the ACA's work shapes), each in longest-processing-time-first order (m + n
// descending; in the half- and quarter-warp shapes then by rank_order; tree
// order on ties); the order comes from one sort of packed 64-bit keys so that
// each FarBlock is written once.

// Row partition of a block list (rows in cluster order): part boundaries
// only where no block's row range is cut, each part's estimated cost as
// close as the boundaries allow to 1/n_parts of the total.  Cost of a dense
// block m n entries, of an admissible block (m + n) rank_est (the entries
// its ACA requests at that rank); a block's cost is spread evenly over its
// rows.  The paper's multi-GPU assembly splits the block list evenly between
// its GPUs (Sec. 4.1); this generalises that to a cost-balanced split of the
// block rows, so that each part owns whole rows of the matrix.
constexpr double kPartRankEst = 10.0;  // typical ACA rank of the workloads (eps 1e-4 .. 1e-5)

void partition_rows(const int64_t *blocks, int64_t nb, int64_t n, int32_t parts, double rank_est,
                    int64_t *bounds)
{
    std::vector<int64_t> cross(n + 2, 0);
    std::vector<double> cost(n + 1, 0.0);
    for (int64_t b = 0; b < nb; ++b) {
        const int64_t *r = blocks + 5 * b;
        const int64_t tb = r[0], te = r[1], m = r[1] - r[0], nn = r[3] - r[2];
        if (m <= 0) continue;
        if (te - tb > 1) {  // rows strictly inside (tb, te) may not be boundaries
            cross[tb + 1] += 1;
            cross[te] -= 1;
        }
        const double c = r[4] ? (double)(m + nn) * rank_est : (double)m * (double)nn;
        cost[tb] += c / m;
        cost[te] -= c / m;
    }
    // per-row cost and prefix sums
    std::vector<double> pre(n + 1, 0.0);
    double run = 0.0;
    int64_t cr = 0;
    std::vector<char> ok(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
        run += cost[i];
        pre[i + 1] = pre[i] + run;
        cr += cross[i];
        ok[i] = cr == 0;
    }
    ok[0] = ok[n] = 1;
    bounds[0] = 0;
    bounds[parts] = n;
    const double total = pre[n];
    int64_t prev = 0;
    for (int32_t p = 1; p < parts; ++p) {
        const double target = total * p / parts;
        int64_t best = prev;
        double bd = std::fabs(pre[prev] - target);
        for (int64_t r = prev; r <= n; ++r) {
            if (!ok[r]) continue;
            const double d = std::fabs(pre[r] - target);
            if (d < bd) {
                bd = d;
                best = r;
            }
            if (pre[r] > target) break;
        }
        bounds[p] = best;
        prev = best;
    }
}

// Keeps the blocks whose row cluster lies in [H.row_b, H.row_e).
void restrict_rows(bem_hmat_s &H)
{
    std::vector<BlockH> keep;
    for (const BlockH &B : H.blocks) {
        const Cluster &T = H.cl[B.tau];
        if (T.b >= H.row_b && T.e <= H.row_e) keep.push_back(B);
        else if (T.e > H.row_b && T.b < H.row_e)
            throw std::invalid_argument("the row range cuts the rows of a block");
    }
    H.blocks.swap(keep);
}

// Order of an admissible block among those of its size in the half- and
// quarter-warp shapes, whose 2 or 4 blocks per warp run in step until the
// highest-rank one ends: a 12-bit bucket of the centre distance of the two
// cluster boxes over the sum of their diameters, which falls as the ACA rank
// grows (on the L6 sphere, correlation -0.57 to -0.72 with the ranks of SLP
// and DLP blocks), so that blocks of like rank share a warp, the likely
// higher ranks first.
static uint64_t rank_order(const Cluster &T, const Cluster &S)
{
    double c2 = 0.0, dt = 0.0, ds = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double c = 0.5 * ((T.box[a] + T.box[a + 3]) - (S.box[a] + S.box[a + 3]));
        const double et = T.box[a + 3] - T.box[a], es = S.box[a + 3] - S.box[a];
        c2 += c * c;
        dt += et * et;
        ds += es * es;
    }
    const double den = std::sqrt(dt) + std::sqrt(ds);
    const double r = den > 0.0 ? std::sqrt(c2) / den : 8.0;
    return (uint64_t)std::min(4095.0, std::floor(r * 512.0));
}

void build_lists(bem_hmat_s &H)
{
    PhaseTrace trace("lists");
    const bem_mesh_s &M = *H.mesh;
    const int64_t nb = (int64_t)H.blocks.size(), nt = M.nt;
    if (nb >= (int64_t(1) << 32) || nt >= (int64_t(1) << 29))
        throw std::runtime_error("problem too large for the block-list keys");
    constexpr uint64_t kSizeMask = (uint64_t(1) << 29) - 1;
    // near blocks (tree order, consecutive dense storage) and keys of the
    // admissible blocks, in block chunks on the host threads, joined in order
    constexpr int64_t kBlkChunk = 16384;
    const int64_t nbc = (nb + kBlkChunk - 1) / kBlkChunk;
    struct BlkPart {
        std::vector<NearBlock> near;
        std::vector<int64_t> near_id;
        std::vector<uint64_t> key;
        int64_t elems = 0, ncls[5] = {0, 0, 0, 0, 0};
    };
    std::vector<BlkPart> bp(nbc);
    parallel_tasks(nbc, [&](int64_t ck) {
        // built in locals and moved in at the end: the parts of neighbouring
        // chunks share cache lines
        BlkPart P;
        for (int64_t b = ck * kBlkChunk, be = std::min(nb, b + kBlkChunk); b < be; ++b) {
            const Cluster &T = H.cl[H.blocks[b].tau], &S = H.cl[H.blocks[b].sigma];
            const int64_t m = T.e - T.b, n = S.e - S.b;
            if (!H.blocks[b].adm) {
                P.near.push_back({T.b, T.e, S.b, S.e, P.elems});   // offset within the chunk
                P.near_id.push_back(b);
                P.elems += m * n * H.dofs * H.dofs;
            } else {
                // work shape (AcaShape): CTA, warp, half warp, quarter warp,
                // lane; piecewise linear blocks take CTAs and warps only
                const int64_t mx = std::max(m, n) * H.dofs;
                uint64_t cls;
                if (mx > H.small_max) cls = kShapeCta;
                else if (mx <= H.tiny_max) cls = kShapeLane;
                else if (H.dofs != 1 || mx > kSub16Max) cls = kShapeWarp;
                else if (mx > kSub8Max) cls = kShapeHalf;
                else cls = kShapeQuarter;
                ++P.ncls[cls];
                uint64_t sz = kSizeMask - (uint64_t)(m + n);
                if (cls == kShapeHalf || cls == kShapeQuarter) sz = (uint64_t)(255 - (m + n)) << 12 | rank_order(T, S);
                P.key.push_back(cls << 61 | sz << 32 | (uint64_t)b);
            }
        }
        bp[ck] = std::move(P);
    });
    trace.mark("classify");
    // the parts in order: their offsets first, then the copies on the threads
    std::vector<int64_t> at_near(nbc + 1, 0), at_key(nbc + 1, 0), at_elems(nbc + 1, 0);
    int64_t ncls[5] = {0, 0, 0, 0, 0};
    for (int64_t ck = 0; ck < nbc; ++ck) {
        at_near[ck + 1] = at_near[ck] + (int64_t)bp[ck].near.size();
        at_key[ck + 1] = at_key[ck] + (int64_t)bp[ck].key.size();
        at_elems[ck + 1] = at_elems[ck] + bp[ck].elems;
        for (int c = 0; c < 5; ++c) ncls[c] += bp[ck].ncls[c];
    }
    H.near.clear();
    H.near.resize(at_near[nbc]);
    H.near_block_id.clear();
    H.near_block_id.resize(at_near[nbc]);
    std::vector<uint64_t, NoInit<uint64_t>> key(at_key[nbc]);
    parallel_tasks(nbc, [&](int64_t ck) {
        const BlkPart &P = bp[ck];
        for (size_t q = 0; q < P.near.size(); ++q) {
            NearBlock N = P.near[q];
            N.off += at_elems[ck];
            H.near[at_near[ck] + q] = N;
            H.near_block_id[at_near[ck] + q] = P.near_id[q];
        }
        std::copy(P.key.begin(), P.key.end(), key.begin() + at_key[ck]);
    });
    H.near_total = at_elems[nbc];
    trace.mark("join");
    // the keys were made in increasing block order, so a stable sort on the
    // upper 32 bits (class, size, rank order) alone orders them fully: LSD passes of 8
    // bits, each with digit counts per chunk on the threads, the offsets in
    // (digit, chunk) order and a stable scatter per chunk; a pass whose keys
    // all share their digit is skipped
    {
        const int64_t nk = (int64_t)key.size();
        const int64_t nck = std::max<int64_t>(1, std::min<int64_t>(64, nk / 16384));
        const int64_t per = (nk + nck - 1) / nck;
        std::vector<uint64_t, NoInit<uint64_t>> tmp(nk);
        std::vector<std::array<int64_t, 256>> cnt(nck);
        for (int pass = 0; pass < 4 && nk > 1; ++pass) {
            const int sh = 32 + 8 * pass;
            parallel_tasks(nck, [&](int64_t ck) {
                std::array<int64_t, 256> &c = cnt[ck];
                c.fill(0);
                for (int64_t i = ck * per, ie = std::min(nk, i + per); i < ie; ++i)
                    ++c[(key[i] >> sh) & 0xffu];
            });
            int used = 0;
            for (int d = 0; d < 256; ++d) {
                int64_t tot = 0;
                for (int64_t ck = 0; ck < nck; ++ck) tot += cnt[ck][d];
                used += tot > 0;
            }
            if (used <= 1) continue;
            int64_t run = 0;
            for (int d = 0; d < 256; ++d)
                for (int64_t ck = 0; ck < nck; ++ck) {
                    const int64_t v = cnt[ck][d];
                    cnt[ck][d] = run;
                    run += v;
                }
            parallel_tasks(nck, [&](int64_t ck) {
                std::array<int64_t, 256> pos = cnt[ck];
                for (int64_t i = ck * per, ie = std::min(nk, i + per); i < ie; ++i)
                    tmp[pos[(key[i] >> sh) & 0xffu]++] = key[i];
            });
            key.swap(tmp);
        }
    }
    trace.mark("sort");
    H.far.resize(key.size());
    H.far_block_id.resize(key.size());
    H.max_m_big = H.max_m_small = 0;
    const int64_t nfar = (int64_t)key.size();
    const int64_t nfc = (nfar + kBlkChunk - 1) / kBlkChunk;
    std::vector<int64_t> mbig(nfc, 0), msmall(nfc, 0);
    std::vector<char> low_rule(nfc, 0);  // some block of the chunk has a lower-order rule
    parallel_tasks(nfc, [&](int64_t ck) {
        bool low = false;
        int64_t mb = 0, ms = 0;
        for (int64_t f = ck * kBlkChunk, fe = std::min(nfar, f + kBlkChunk); f < fe; ++f) {
            const int64_t b = (int64_t)(key[f] & 0xffffffffu);
            const Cluster &T = H.cl[H.blocks[b].tau], &S = H.cl[H.blocks[b].sigma];
            FarBlock &F = H.far[f];
            std::memset(&F, 0, sizeof(F));
            F.tb = T.b;
            F.te = T.e;
            F.sb = S.b;
            F.se = S.e;
            F.rule = H.dofs == 1 ? block_rule(T, S, H.rho3, H.rho1) : kRule6;
            low |= F.rule != kRule6;
            H.far_block_id[f] = b;
            if (f < ncls[kShapeCta]) mb = std::max(mb, T.e - T.b);
            else if (f < ncls[kShapeCta] + ncls[kShapeWarp]) ms = std::max(ms, T.e - T.b);
        }
        mbig[ck] = mb;
        msmall[ck] = ms;
        low_rule[ck] = low;
    });
    for (int64_t ck = 0; ck < nfc; ++ck) {
        H.max_m_big = std::max(H.max_m_big, mbig[ck]);
        H.max_m_small = std::max(H.max_m_small, msmall[ck]);
    }
    for (int c = 0; c < 5; ++c) H.nshape[c] = ncls[c];
    H.has_rules = false;
    for (char c : low_rule) H.has_rules |= c != 0;
    trace.mark("far");

    // leaves sorted by row start, and the leaf of every cluster-order row
    std::vector<std::pair<int64_t, int64_t>> lr;
    for (const Cluster &C : H.cl)
        if (C.left < 0) lr.push_back({C.b, C.e});
    std::sort(lr.begin(), lr.end());
    const int64_t nleaf = (int64_t)lr.size();
    std::vector<int64_t> leaf_of(nt, -1);
    H.leaf_rows.resize(2 * nleaf);
    for (int64_t l = 0; l < nleaf; ++l) {
        H.leaf_rows[2 * l] = lr[l].first;
        H.leaf_rows[2 * l + 1] = lr[l].second;
        for (int64_t p = lr[l].first; p < lr[l].second; ++p) leaf_of[p] = l;
    }
    trace.mark("leaves");
    // per leaf, the blocks whose row range contains it: far blocks in list
    // order as f, then near blocks in tree order as -1 - q (CSR).  A block
    // covers a leaf exactly when its row cluster is the leaf's cluster or an
    // ancestor of it: every cluster lists its own blocks, and each leaf (on
    // the threads) copies the lists along its path to the root into its slot
    // and sorts them there (the indices are distinct, so the sorted slot is
    // the list order).
    const int64_t ncl = (int64_t)H.cl.size();
    const int64_t nfar_b = (int64_t)H.far.size(), nnear_b = (int64_t)H.near.size();
    std::vector<int64_t> parent(ncl, -1), leaf_cl(nleaf, -1);
    for (int64_t c = 0; c < ncl; ++c) {
        const Cluster &C = H.cl[c];
        if (C.left >= 0) {
            parent[C.left] = c;
            parent[C.right] = c;
        } else {
            leaf_cl[leaf_of[C.b]] = c;
        }
    }
    // row cluster of every far and near block, then a CSR per cluster
    std::vector<int32_t, NoInit<int32_t>> tau_far(nfar_b), tau_near(nnear_b);
    parallel_tasks((nfar_b + 65535) / 65536, [&](int64_t task) {
        for (int64_t f = task * 65536, fe = std::min(nfar_b, f + 65536); f < fe; ++f)
            tau_far[f] = (int32_t)H.blocks[H.far_block_id[f]].tau;
    });
    parallel_tasks((nnear_b + 65535) / 65536, [&](int64_t task) {
        for (int64_t q = task * 65536, qe = std::min(nnear_b, q + 65536); q < qe; ++q)
            tau_near[q] = (int32_t)H.blocks[H.near_block_id[q]].tau;
    });
    // a stable counting sort of the blocks by row cluster, in chunks of the
    // blocks on the host threads: per-chunk counts, offsets in (cluster,
    // chunk) order, and each chunk's blocks scattered in order
    auto cluster_lists = [&](const std::vector<int32_t, NoInit<int32_t>> &tau, std::vector<int64_t> &ptr,
                             std::vector<int64_t, NoInit<int64_t>> &idx) {
        const int64_t n = (int64_t)tau.size();
        const int64_t nck = std::max<int64_t>(1, std::min<int64_t>(8, n / 32768));
        const int64_t per = (n + nck - 1) / nck;
        std::vector<std::vector<int64_t>> cnt(nck);
        parallel_tasks(nck, [&](int64_t ck) {
            std::vector<int64_t> &c = cnt[ck];
            c.assign(ncl, 0);
            for (int64_t x = ck * per, xe = std::min(n, x + per); x < xe; ++x) ++c[tau[x]];
        });
        ptr.assign(ncl + 1, 0);
        int64_t run = 0;
        for (int64_t c = 0; c < ncl; ++c) {
            ptr[c] = run;
            for (int64_t ck = 0; ck < nck; ++ck) {
                const int64_t v = cnt[ck][c];
                cnt[ck][c] = run;
                run += v;
            }
        }
        ptr[ncl] = run;
        idx.resize(n);
        parallel_tasks(nck, [&](int64_t ck) {
            std::vector<int64_t> &pos = cnt[ck];
            for (int64_t x = ck * per, xe = std::min(n, x + per); x < xe; ++x) idx[pos[tau[x]]++] = x;
        });
    };
    std::vector<int64_t> cf_ptr, cn_ptr;
    std::vector<int64_t, NoInit<int64_t>> cf_idx, cn_idx;
    cluster_lists(tau_far, cf_ptr, cf_idx);
    cluster_lists(tau_near, cn_ptr, cn_idx);
    trace.mark("items_count");
    H.leaf_ptr.assign(nleaf + 1, 0);
    std::vector<int64_t> leaf_nfar(nleaf);
    parallel_tasks((nleaf + 1023) / 1024, [&](int64_t task) {
        for (int64_t l = task * 1024, le = std::min(nleaf, l + 1024); l < le; ++l) {
            int64_t nf = 0, nn = 0;
            for (int64_t c = leaf_cl[l]; c >= 0; c = parent[c]) {
                nf += cf_ptr[c + 1] - cf_ptr[c];
                nn += cn_ptr[c + 1] - cn_ptr[c];
            }
            leaf_nfar[l] = nf;
            H.leaf_ptr[l + 1] = nf + nn;
        }
    });
    for (int64_t l = 0; l < nleaf; ++l) H.leaf_ptr[l + 1] += H.leaf_ptr[l];
    H.leaf_items.resize(H.leaf_ptr[nleaf]);
    trace.mark("items_offsets");
    parallel_tasks((nleaf + 255) / 256, [&](int64_t task) {
        for (int64_t l = task * 256, le = std::min(nleaf, l + 256); l < le; ++l) {
            int64_t *const out = H.leaf_items.data() + H.leaf_ptr[l];
            int64_t *w = out;
            for (int64_t c = leaf_cl[l]; c >= 0; c = parent[c])
                w = std::copy(cf_idx.begin() + cf_ptr[c], cf_idx.begin() + cf_ptr[c + 1], w);
            std::sort(out, w);
            int64_t *const near0 = w;
            for (int64_t c = leaf_cl[l]; c >= 0; c = parent[c])
                w = std::copy(cn_idx.begin() + cn_ptr[c], cn_idx.begin() + cn_ptr[c + 1], w);
            std::sort(near0, w);
            for (int64_t *x = near0; x < w; ++x) *x = -1 - *x;
        }
    });
    trace.mark("leaf_far_items");
    // near blocks per row leaf, by column start (the columns of one leaf's
    // blocks are disjoint, so the starts are distinct), for the touching
    // pairs: the near part of each leaf's item list, sorted by column start
    std::vector<int64_t> nptr(nleaf + 1, 0);
    for (int64_t l = 0; l < nleaf; ++l)
        nptr[l + 1] = nptr[l] + (H.leaf_ptr[l + 1] - H.leaf_ptr[l] - leaf_nfar[l]);
    std::vector<int64_t, NoInit<int64_t>> nq(nptr[nleaf]), nsb(nptr[nleaf]);
    parallel_tasks((nleaf + 1023) / 1024, [&](int64_t task) {
        for (int64_t l = task * 1024, le = std::min(nleaf, l + 1024); l < le; ++l) {
            const int64_t *it = H.leaf_items.data() + H.leaf_ptr[l] + leaf_nfar[l];
            for (int64_t i = nptr[l]; i < nptr[l + 1]; ++i) nq[i] = -1 - *it++;
            std::sort(nq.begin() + nptr[l], nq.begin() + nptr[l + 1],
                      [&](int64_t a, int64_t b) { return H.near[a].sb < H.near[b].sb; });
            for (int64_t i = nptr[l]; i < nptr[l + 1]; ++i) nsb[i] = H.near[nq[i]].sb;
        }
    });
    trace.mark("leaf_near_items");
    // singular pairs of the near field, with their place in the dense blocks
    for (int c = 0; c < 3; ++c) {
        H.sing[c].clear();
        H.singl[c].clear();
    }
    // rows in chunks on the host threads, each chunk's pairs in row order,
    // the chunks in order (the sequential order): the chunks count their
    // pairs per case, the prefix over the chunks gives each its first slot,
    // and the chunks write their pairs into the final lists.
    // P0 vertex-adjacent pairs are listed once, as (lower, higher) cluster
    // position, with the offsets of both entries (-1 for an entry whose row
    // another part of a row partition holds): the two share the rule's
    // nodes (k_singular, SYM), and each entry's value is the same whatever
    // the partition.
    const bool vsym = H.dofs == 1;
    auto mirrored = [&](int64_t p, int64_t q) { return q >= H.row_b && q < H.row_e && q < p; };
    constexpr int64_t kRowChunk = 8192;
    const int64_t nchunk = (nt + kRowChunk - 1) / kRowChunk;
    std::vector<std::array<int64_t, 3>> at(nchunk + 1, std::array<int64_t, 3>{0, 0, 0});
    parallel_tasks(nchunk, [&](int64_t ck) {
        std::array<int64_t, 3> cnt{0, 0, 0};
        for (int64_t p = std::max(ck * kRowChunk, H.row_b),
                     pe = std::min({nt, ck * kRowChunk + kRowChunk, H.row_e});
             p < pe; ++p) {
            const int32_t t = H.perm[p];
            for (int64_t a = M.adj_ptr[t]; a < M.adj_ptr[t + 1]; ++a) {
                const int c = M.adj_case[a] - 1;
                if (vsym && c == 0 && mirrored(p, H.iperm[M.adj_tri[a]])) continue;
                ++cnt[c];
            }
        }
        at[ck + 1] = cnt;
    });
    for (int64_t ck = 0; ck < nchunk; ++ck)
        for (int c = 0; c < 3; ++c) at[ck + 1][c] += at[ck][c];
    for (int c = 0; c < 3; ++c) {
        if (H.dofs == 1) H.sing[c].resize(at[nchunk][c]);
        else H.singl[c].resize(at[nchunk][c]);
    }
    H.sing_t.resize(vsym ? at[nchunk][0] : 0);
    trace.mark("singular_count");
    // the near block of row leaf l whose column range holds column q
    // each leaf's own block (columns the leaf's rows), where most touching
    // pairs lie: found without a search when the column falls in the leaf
    std::vector<int64_t> diag(nleaf, -1);
    parallel_tasks((nleaf + 1023) / 1024, [&](int64_t task) {
        for (int64_t l = task * 1024, le = std::min(nleaf, l + 1024); l < le; ++l) {
            const int64_t *b0 = nsb.data() + nptr[l], *b1 = nsb.data() + nptr[l + 1];
            const int64_t *it = std::lower_bound(b0, b1, H.leaf_rows[2 * l]);
            if (it != b1 && *it == H.leaf_rows[2 * l]) {
                const int64_t id = nq[nptr[l] + (it - b0)];
                if (H.near[id].se == H.leaf_rows[2 * l + 1]) diag[l] = id;
            }
        }
    });
    auto near_of = [&](int64_t l, int64_t q) -> const NearBlock & {
        if (diag[l] >= 0 && q >= H.leaf_rows[2 * l] && q < H.leaf_rows[2 * l + 1]) return H.near[diag[l]];
        const int64_t *b0 = nsb.data() + nptr[l], *b1 = nsb.data() + nptr[l + 1];
        const int64_t *it = std::upper_bound(b0, b1, q);
        if (it == b0) throw std::runtime_error("touching pair outside the near field");
        const NearBlock &N = H.near[nq[nptr[l] + (it - 1 - b0)]];
        if (q >= N.se) throw std::runtime_error("touching pair outside the near field");
        return N;
    };
    parallel_tasks(nchunk, [&](int64_t ck) {
        std::array<int64_t, 3> pos = at[ck];
        for (int64_t p = std::max(ck * kRowChunk, H.row_b),
                     pe = std::min({nt, ck * kRowChunk + kRowChunk, H.row_e});
             p < pe; ++p) {
            const int32_t t = H.perm[p];
            const int64_t l = leaf_of[p];
            for (int64_t a = M.adj_ptr[t]; a < M.adj_ptr[t + 1]; ++a) {
                const int32_t u = M.adj_tri[a];
                const int64_t q = H.iperm[u];
                const int c = M.adj_case[a] - 1;
                if (vsym && c == 0 && mirrored(p, q)) continue;  // listed from row q
                // near block of this row leaf whose column range holds q
                const NearBlock &N = near_of(l, q);
                if (H.dofs == 1) {
                    // column-major block
                    const int64_t dest = N.off + (q - N.sb) * (N.te - N.tb) + (p - N.tb);
                    if (c == 0 && q < p) {
                        // row q lies in another part: the pair (q, p) writes
                        // only its transposed entry, this row's
                        H.sing_t[pos[c]] = dest;
                        H.sing[c][pos[c]++] = {u, t, -1};
                        continue;
                    }
                    if (c == 0) {
                        int64_t d2 = -1;
                        if (q >= H.row_b && q < H.row_e) {  // (q, p) is a row of this matrix
                            const NearBlock &N2 = near_of(leaf_of[q], p);
                            d2 = N2.off + (p - N2.sb) * (N2.te - N2.tb) + (q - N2.tb);
                        }
                        H.sing_t[pos[c]] = d2;
                    }
                    H.sing[c][pos[c]++] = {t, u, dest};
                } else {
                    // local (0, 0) of the pair in the column-major block of
                    // 3m x 3n dofs: rows step by 1, columns by 3m
                    const int64_t ld = 3 * (N.te - N.tb);
                    const int64_t dest = N.off + 3 * (q - N.sb) * ld + 3 * (p - N.tb);
                    H.singl[c][pos[c]++] = {t, u, dest, 1, (int32_t)ld};
                }
            }
        }
    });
    for (int c = 0; c < 3; ++c)
        H.sing_entries[c] = H.dofs == 1 ? (int64_t)H.sing[c].size() : (int64_t)H.singl[c].size();
    if (vsym) {
        H.sing_entries[0] = 0;
        for (size_t i = 0; i < H.sing_t.size(); ++i)
            H.sing_entries[0] += (H.sing[0][i].dest >= 0) + (H.sing_t[i] >= 0);
    }
    trace.mark("singular");
    trace.mark("join_singular");
    if (H.dofs == 3) {
        // every list in dof units: ranges times three
        for (NearBlock &N : H.near) {
            N.tb *= 3;
            N.te *= 3;
            N.sb *= 3;
            N.se *= 3;
        }
        for (FarBlock &F : H.far) {
            F.tb *= 3;
            F.te *= 3;
            F.sb *= 3;
            F.se *= 3;
        }
        for (int64_t &r : H.leaf_rows) r *= 3;
        H.max_m_big *= 3;
        H.max_m_small *= 3;
        H.dperm.resize(3 * nt);
        for (int64_t p = 0; p < nt; ++p)
            for (int a = 0; a < 3; ++a) H.dperm[3 * p + a] = 3 * H.perm[p] + a;
    }
    H.ndof = H.dofs * nt;
    if (H.space == BEM_P1) {
        // vertex -> its DP1 dofs 3 t + a (T[t][a] = v), in increasing dof order
        const int64_t nv = M.nv;
        H.vptr.assign(nv + 1, 0);
        for (int64_t q = 0; q < 3 * nt; ++q) ++H.vptr[M.T[q] + 1];
        for (int64_t v = 0; v < nv; ++v) H.vptr[v + 1] += H.vptr[v];
        H.vdof.resize(3 * nt);
        std::vector<int64_t> fill(H.vptr.begin(), H.vptr.end() - 1);
        for (int64_t q = 0; q < 3 * nt; ++q) H.vdof[fill[M.T[q]]++] = (int32_t)q;
    }
}

void upload_tree(bem_hmat_s &H, cudaStream_t st)
{
    H.d_perm.upload(H.perm, st);
    H.d_near.upload(H.near, st);
    H.d_far.upload(H.far, st);
    H.d_chunks.alloc(H.far.size() * sizeof(FarChunks), st);
    for (int c = 0; c < 3; ++c) H.d_sing[c].upload(H.sing[c], st);
    H.d_sing_t.upload(H.sing_t, st);
    if (H.dofs == 3) {
        H.d_dperm.upload(H.dperm, st);
        for (int c = 0; c < 3; ++c) H.d_singl[c].upload(H.singl[c], st);
    }
    if (H.space == BEM_P1) {
        H.d_vptr.upload(H.vptr, st);
        H.d_vdof.upload(H.vdof, st);
    }
    H.d_leaf_rows.upload(H.leaf_rows, st);
    H.d_leaf_ptr.upload(H.leaf_ptr, st);
    H.d_leaf_items.upload(H.leaf_items, st);
    H.long_ids.clear();
    for (size_t b = 0; b < H.far.size(); ++b)
        if (H.far[b].se - H.far[b].sb > kMatvecLongCol) H.long_ids.push_back((int64_t)b);
    H.d_long.upload(H.long_ids, st);
    H.d_long_off.alloc((H.long_ids.size() + 1) * sizeof(int64_t), st);
    DeviceConsts &D = device_consts();
    H.geom.build(H.mesh->dV.as<double>(), H.mesh->dT.as<int32_t>(), H.d_perm.as<int32_t>(),
                 H.mesh->nt, D.rule, st);
    H.d_poolhdr.alloc(sizeof(Pool), st);
    H.d_queue.alloc(sizeof(AcaQueue), st);
    H.d_toff.alloc((H.far.size() + 1) * sizeof(int64_t), st);
    H.d_tiles.alloc(aca_finish_tiles((int64_t)H.far.size()) * sizeof(int64_t), st);
    H.d_acastats.alloc(sizeof(AcaStats), st);
    H.d_job.alloc(sizeof(AcaJob), st);
    CU(cudaStreamSynchronize(st));
}

}  // namespace

extern "C" {

}  // extern "C"

namespace bem {

// Tree build on the host, uploads and geometry on stream st (none for
// st == kHostOnly).
int hmat_build_tree_impl(bem_mesh mesh, int32_t leaf_size, double eta, cudaStream_t st,
                         bem_hmat *out, int32_t space, int32_t n_parts, int32_t part)
{
    return guarded([&]() -> int {
        if (!out) return fail(BEM_E_ARG, "out is null");
        *out = nullptr;
        if (!mesh) return fail(BEM_E_ARG, "null mesh");
        if (leaf_size < 1) return fail(BEM_E_ARG, "leaf_size must be >= 1");
        if (!(eta > 0) || !std::isfinite(eta)) return fail(BEM_E_ARG, "eta must be > 0");
        if (space != BEM_P0 && space != BEM_DP1 && space != BEM_P1)
            return fail(BEM_E_ARG, "bad space");
        double t0 = now_ms();
        auto H = std::make_unique<bem_hmat_s>();
        H->mesh = mesh;
        H->leaf = leaf_size;
        H->eta = eta;
        H->space = space;
        H->dofs = space == BEM_P0 ? 1 : 3;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            H->small_max = g_tuning.warp_max_rows;
            H->tiny_max = H->dofs == 1 ? g_tuning.lane_max_rows : 0;
            H->rho3 = H->dofs == 1 ? g_quad.rho3 : 0.0;
            H->rho1 = H->dofs == 1 ? g_quad.rho1 : 0.0;
        }
        if (n_parts < 1 || part < 0 || part >= n_parts)
            return fail(BEM_E_ARG, "bad part of the row partition");
        if (n_parts > 1 && space != BEM_P0)
            return fail(BEM_E_ARG, "row partitions are for P0 handles");
        build_clusters(*H);
        const double t1 = now_ms();
        build_blocks(*H);
        H->row_b = 0;
        H->row_e = mesh->nt;
        if (n_parts > 1) {
            // this part's block rows: the partition of the whole block list
            std::vector<int64_t> bl(5 * H->blocks.size()), bounds(n_parts + 1);
            for (size_t b = 0; b < H->blocks.size(); ++b) {
                const Cluster &T = H->cl[H->blocks[b].tau], &S = H->cl[H->blocks[b].sigma];
                int64_t *r = bl.data() + 5 * b;
                r[0] = T.b;
                r[1] = T.e;
                r[2] = S.b;
                r[3] = S.e;
                r[4] = H->blocks[b].adm ? 1 : 0;
            }
            partition_rows(bl.data(), (int64_t)H->blocks.size(), mesh->nt, n_parts, kPartRankEst,
                           bounds.data());
            H->row_b = bounds[part];
            H->row_e = bounds[part + 1];
            restrict_rows(*H);
        }
        const double t2 = now_ms();
        build_lists(*H);
        const double t3 = now_ms();
        if (st != kHostOnly) upload_tree(*H, st);
        H->t_tree = now_ms() - t0;
        H->t_clusters = t1 - t0;
        H->t_blocks = t2 - t1;
        H->t_lists = t3 - t2;
        H->t_upload = H->t_tree - (t3 - t0);
        ++mesh->hmat_refs;
        *out = H.release();
        return BEM_OK;
    });
}

// Device part of an H-matrix built with kHostOnly.
int hmat_upload(bem_hmat H, cudaStream_t st)
{
    return guarded([&]() -> int {
        upload_tree(*H, st);
        return BEM_OK;
    });
}

// Device bytes an assembly of this H-matrix holds (geometry, tree arrays,
// dense blocks, factor pool of four 4-column chunks per admissible block, and
// the product buffers), for admission control.
int64_t hmat_device_bytes(bem_hmat H, bool cplx)
{
    const int64_t nt = H->mesh->nt, esz = cplx ? 16 : 8;
    int64_t sum_mn = 0;
    for (const FarBlock &F : H->far) sum_mn += (F.te - F.tb) + (F.se - F.sb);
    int64_t geom = 2 * (nt * (12 + 72 + 24 + 8 + 144) + (nt + 31) / 32 * 32 * 128);  // mesh + cluster order
    int64_t tree = (int64_t)(H->near.size() * sizeof(NearBlock) +
                             H->far.size() * (sizeof(FarBlock) + sizeof(FarChunks))) +
                   (int64_t)(H->sing[0].size() + H->sing[1].size() + H->sing[2].size()) * 16 +
                   (int64_t)H->sing_t.size() * 8 +
                   (int64_t)(H->leaf_items.size() + H->leaf_ptr.size() + H->leaf_rows.size()) * 8 +
                   nt * 4 + (int64_t)H->far.size() * 8 * 2;
    int64_t pool = (sum_mn * KCHUNK * 4 + 1024) * esz;
    int64_t vecs = 5 * nt * esz;
    return geom + tree + H->near_total * esz + pool + vecs;
}

void hmat_free_synced(bem_hmat H)
{
    --H->mesh->hmat_refs;
    delete H;
}

}  // namespace bem

namespace bem {

// ---- stages of an assembly (hmat_assemble; the request server's launches
// over several H-matrices) ---------------------------------------------------

// Checks the arguments, records the key, allocates the near-field buffer and
// sizes the factor pool (H->pool_want); nothing is launched.
int assemble_begin(bem_hmat H, int32_t op, double k, double aca_eps, int32_t prec, cudaStream_t st)
{
    if (!H) return fail(BEM_E_ARG, "null hmat");
    if (op < 0 || op > 3) return fail(BEM_E_ARG, "bad op");
    if (op == BEM_HYPS && H->space != BEM_P1)
        return fail(BEM_E_ARG, "the hypersingular operator needs a BEM_P1 handle");
    if (prec != BEM_FP64 && prec != BEM_MIXED && prec != BEM_MIXED_SP) return fail(BEM_E_ARG, "bad prec");
    if (prec == BEM_MIXED_SP && H->dofs != 1)
        return fail(BEM_E_ARG, "BEM_MIXED_SP applies to P0 handles only");
    if (!(aca_eps > 0) || !std::isfinite(aca_eps)) return fail(BEM_E_ARG, "aca_eps must be > 0");
    if (!std::isfinite(k)) return fail(BEM_E_ARG, "bad k");
    const bool cplx = k != 0.0;
    const size_t esz = cplx ? 16 : 8;
    H->assembled = false;
    H->op = op;
    H->k = k;
    H->eps = aca_eps;
    H->prec = prec;
    H->cplx = cplx;
    if (!H->ev[0])
        for (auto &e : H->ev) CU(cudaEventCreate(&e));
    if (!H->pin_pool) {
        static_assert(sizeof(Pool) <= kPinSlot && sizeof(AcaStats) <= kPinSlot &&
                          sizeof(AcaJob) <= kPinSlot, "pinned slots");
        H->pin_pool = (Pool *)pinned_slot();
        H->pin_stats = (AcaStats *)pinned_slot();
        H->pin_job = (AcaJob *)pinned_slot();
        if (!H->pin_pool || !H->pin_stats || !H->pin_job)
            return fail(BEM_E_OOM, "page-locked host memory for the readbacks");
    }
    if (H->d_near_data.bytes < (size_t)H->near_total * esz)
        H->d_near_data.alloc(H->near_total * esz, st);
    int64_t sum_mn = 0;
    for (const FarBlock &F : H->far) sum_mn += (F.te - F.tb) + (F.se - F.sb);
    // factor pool: room for four chunks per admissible block, capped by
    // what the device has free (less a margin for the product buffers);
    // one chunk per block is the least that can work
    int64_t want = sum_mn * KCHUNK * 4 + 1024;
    {
        size_t fr = 0, tot = 0;
        // blocks cached in the library's pool are not free to the sizing:
        // give them back first when the wish would not fit otherwise
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess &&
            (double)want * esz > (double)fr + (double)H->d_pool.bytes - 4.0 * (1 << 30)) {
            CU(cudaStreamSynchronize(st));
            pool_trim();
        }
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
            const double margin = 4.0 * (1 << 30) + 17.0 * H->ndof * esz;
            const int64_t avail =
                (int64_t)(((double)fr + (double)H->d_pool.bytes - margin) / (double)esz);
            want = std::min(want, avail);
            if (want < sum_mn * KCHUNK + 1024)
                return fail(BEM_E_OOM, "not enough device memory for one " +
                                           std::to_string(KCHUNK) + "-column chunk per block");
        }
    }
    H->pool_want = std::max(want, H->pool_elems);
    return BEM_OK;
}

// Allocates the factor pool at H->pool_want elements and uploads the
// matrix's ACA job (stream-ordered before the launches that follow on st).
void assemble_pool(bem_hmat H, cudaStream_t st)
{
    const size_t esz = H->cplx ? 16 : 8;
    if (H->d_pool.bytes < (size_t)H->pool_want * esz) H->d_pool.alloc((size_t)H->pool_want * esz, st);
    H->pool_elems = H->pool_want;
    *H->pin_job = AcaJob{H->geom.g, H->d_far.as<FarBlock>(), H->d_chunks.as<FarChunks>(),
                         H->d_pool.p, H->d_poolhdr.as<Pool>(), H->k, H->eps,
                         (int64_t)H->far.size()};
    CU(cudaMemcpyAsync(H->d_job.p, H->pin_job, sizeof(AcaJob), cudaMemcpyHostToDevice, st));
}

static void record(cudaEvent_t e, cudaStream_t st, bool capturing)
{
    if (capturing) CU(cudaEventRecordWithFlags(e, st, cudaEventRecordExternal));
    else CU(cudaEventRecord(e, st));
}

// Pool header, queue and totals reset; near field: regular pairs, then the
// touching pairs (FP64).  Events 0 (start), 3 (after the regular pairs) and
// 1 (end of the near field).
static void enqueue_reset(bem_hmat H, cudaStream_t st, bool capturing)
{
    record(H->ev[0], st, capturing);
    CU(launch_aca_reset(H->d_poolhdr.as<Pool>(), (unsigned long long)H->pool_elems,
                        H->d_queue.as<AcaQueue>(), H->d_acastats.as<AcaStats>(), st));
}

static void enqueue_near_field(bem_hmat H, cudaStream_t st, bool capturing)
{
    DeviceConsts &D = device_consts();
    const int aop = H->op == BEM_HYPS ? BEM_SLP : H->op;
    const double k = H->k;
    const int prec = H->prec;
    if (H->dofs == 1) {
        CU(launch_near_regular(H->geom.g, D.rule, aop, k, prec, H->d_near.as<NearBlock>(),
                               (int64_t)H->near.size(), H->d_near_data.p, st));
        record(H->ev[3], st, capturing);
        const SingPair *sp[3] = {H->d_sing[0].as<SingPair>(), H->d_sing[1].as<SingPair>(),
                                 H->d_sing[2].as<SingPair>()};
        int64_t hc[3] = {(int64_t)H->sing[0].size(), (int64_t)H->sing[1].size(),
                         (int64_t)H->sing[2].size()};
        CU(launch_singular(H->mesh->geom.g, D.sing, aop, k, prec, sp, nullptr, hc, H->d_near_data.p, st,
                           nullptr, H->sing_t.empty() ? nullptr : H->d_sing_t.as<int64_t>()));
    } else {
        CU(launch_near_dp1(H->geom.g, D.rule, aop, k, prec, H->d_near.as<NearBlock>(),
                           (int64_t)H->near.size(), H->d_near_data.p, st));
        record(H->ev[3], st, capturing);
        const SingPairL *sp[3] = {H->d_singl[0].as<SingPairL>(), H->d_singl[1].as<SingPairL>(),
                                  H->d_singl[2].as<SingPairL>()};
        int64_t hc[3] = {(int64_t)H->singl[0].size(), (int64_t)H->singl[1].size(),
                         (int64_t)H->singl[2].size()};
        CU(launch_singular_dp1(H->mesh->geom.g, D.sing, aop, k, sp, nullptr, hc, H->d_near_data.p,
                               st));
    }
    record(H->ev[1], st, capturing);
}

// In a captured graph every event record is followed by a kernel: a record
// node with no successor may fire late (two records in a row timed the near
// field as ending after the ACA).
void enqueue_near(bem_hmat H, cudaStream_t st, bool capturing)
{
    enqueue_reset(H, st, capturing);
    enqueue_near_field(H, st, capturing);
}

// The persistent ACA over this matrix's admissible blocks alone.
void enqueue_aca_own(bem_hmat H, cudaStream_t st)
{
    if (H->far.empty()) return;
    DeviceConsts &D = device_consts();
    const int aop = H->op == BEM_HYPS ? BEM_SLP : H->op;
    AcaWork w{H->d_job.as<AcaJob>(), nullptr,
              {H->nshape[0], H->nshape[1], H->nshape[2], H->nshape[3], H->nshape[4]},
              H->max_m_big, H->max_m_small};
    CU(launch_aca(w, D.rule, aop, H->cplx, H->prec, H->d_queue.as<AcaQueue>(), D.num_sms, st,
                  H->dofs, H->has_rules));
}

// Event 2 (end of the ACA), rank prefix sums and totals, and the readbacks
// of the pool header and the totals.
void enqueue_finish(bem_hmat H, cudaStream_t st, bool capturing, bool mark_aca_end)
{
    if (mark_aca_end) record(H->ev[2], st, capturing);
    CU(launch_aca_finish(H->d_far.as<FarBlock>(), H->d_chunks.as<FarChunks>(),
                         (int64_t)H->far.size(), H->d_toff.as<int64_t>(), H->d_tiles.as<int64_t>(),
                         H->d_acastats.as<AcaStats>(), st));
    CU(launch_long_offsets(H->d_far.as<FarBlock>(), H->d_long.as<int64_t>(),
                           (int64_t)H->long_ids.size(), H->d_long_off.as<int64_t>(), st));
    CU(cudaMemcpyAsync(H->pin_pool, H->d_poolhdr.p, sizeof(Pool), cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(H->pin_stats, H->d_acastats.p, sizeof(AcaStats), cudaMemcpyDeviceToHost, st));
}

bool assemble_overflowed(bem_hmat H) { return H->pin_pool && H->pin_pool->overflow; }

bool hmat_has_rules(bem_hmat H) { return H->has_rules; }

int guarded_call(const std::function<int()> &f)
{
    return guarded([&]() -> int { return f(); });
}

// After the stream has synchronised without pool overflow: totals, phase
// times, and the product's buffers.
void assemble_end(bem_hmat H, cudaStream_t st)
{
    const size_t esz = H->cplx ? 16 : 8;
    cudaEvent_t *ev = H->ev;
    const AcaStats ast = *H->pin_stats;
    float tn = 0, tf = 0, tr = 0;
    CU(cudaEventElapsedTime(&tn, ev[0], ev[1]));
    CU(cudaEventElapsedTime(&tf, ev[1], ev[2]));
    CU(cudaEventElapsedTime(&tr, ev[0], ev[3]));
    H->t_near = tn;
    H->t_far = tf;
    H->t_near_reg = tr;
    H->far_entries = (int64_t)ast.entries;
    H->rank_sum = (int64_t)ast.rank_sum;
    H->capped = ast.capped;
    H->rank_min = H->far.empty() ? 0 : ast.rank_min;
    H->rank_max = ast.rank_max;
    H->factor_elems = (int64_t)ast.factor_elems;
    H->k2mn = (int64_t)ast.k2mn;
    H->rank_mn = (int64_t)ast.rank_mn;
    H->far_result_valid = false;
    const int64_t nd = H->ndof;
    if (H->d_xt.bytes < nd * esz) {
        H->d_xt.alloc(nd * esz, st);
        H->d_yt.alloc(nd * esz, st);
    }
    if (H->space == BEM_P1) {
        // transformed vectors of the products: six DP1 vectors in and out
        // (three curl components and three normal components, Eq. (9));
        // one of each for SLP, DLP and ADLP
        const size_t want_v = (size_t)(H->op == BEM_HYPS ? 6 : 1) * nd * esz;
        if (H->d_xs.bytes < want_v) {
            H->d_xs.alloc(want_v, st);
            H->d_ys.alloc(want_v, st);
        }
    }
    if (H->d_tbuf.bytes < (size_t)(H->rank_sum + 1) * esz)
        H->d_tbuf.alloc((size_t)(H->rank_sum + 1) * esz * 5 / 4, st);
    H->assembled = true;
}

// One persistent ACA launch over the admissible blocks of several
// H-matrices (P0, the same operator, precision and number type, all past
// assemble_pool and enqueue_near on st): the blocks of each work shape from
// every matrix, merged longest first, each item naming its matrix's job.
// sm_share < 1 caps the launch's CTAs at that share of the device, so that
// launches on other streams find free SMs while it runs.  pinned (optional):
// page-locked staging of pinned_bytes for the work list, which must stay
// untouched until the stream has run the copies.
int enqueue_aca_fused(const std::vector<bem_hmat> &hs, cudaStream_t st, double sm_share,
                      void *pinned, size_t pinned_bytes)
{
    if (hs.empty()) return BEM_OK;
    DeviceConsts &D = device_consts();
    const bem_hmat H0 = hs[0];
    const int aop = H0->op == BEM_HYPS ? BEM_SLP : H0->op;
    std::vector<AcaJob> jobs;
    struct It {
        int64_t size, item;
    };
    std::vector<It> cls[5];
    int64_t max_big = 0, max_small = 0;
    for (size_t j = 0; j < hs.size(); ++j) {
        const bem_hmat H = hs[j];
        if (H->dofs != 1 || H->op != H0->op || H->cplx != H0->cplx || H->prec != H0->prec ||
            H->has_rules != H0->has_rules)
            return fail(BEM_E_ARG, "fused ACA launch over different kinds of matrices");
        jobs.push_back(*H->pin_job);
        int64_t f = 0;
        for (int c = 0; c < 5; ++c)
            for (int64_t e = f + H->nshape[c]; f < e; ++f) {
                const FarBlock &F = H->far[f];
                cls[c].push_back({(F.te - F.tb) + (F.se - F.sb), ((int64_t)j << kItemShift) | f});
            }
        max_big = std::max(max_big, H->max_m_big);
        max_small = std::max(max_small, H->max_m_small);
    }
    std::vector<int64_t> items;
    for (auto &c : cls) {
        std::stable_sort(c.begin(), c.end(), [](const It &a, const It &b) { return a.size > b.size; });
        for (const It &i : c) items.push_back(i.item);
    }
    if (items.empty()) return BEM_OK;
    const size_t jb = (jobs.size() * sizeof(AcaJob) + 255) / 256 * 256;
    const size_t ib = items.size() * sizeof(int64_t);
    void *buf = nullptr;
    CU(lib_malloc_async(&buf, jb + ib + sizeof(AcaQueue), st));
    char *b = (char *)buf;
    AcaQueue *Q = (AcaQueue *)(b + jb + ib);
    // from page-locked staging if the caller has some (a copy from pageable
    // memory first waits for the stream's pending work)
    const void *src_jobs = jobs.data(), *src_items = items.data();
    if (pinned && pinned_bytes >= jb + ib) {
        std::memcpy(pinned, jobs.data(), jobs.size() * sizeof(AcaJob));
        std::memcpy((char *)pinned + jb, items.data(), ib);
        src_jobs = pinned;
        src_items = (char *)pinned + jb;
    }
    cudaError_t e = cudaMemcpyAsync(b, src_jobs, jobs.size() * sizeof(AcaJob),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + jb, src_items, ib, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(Q, 0, sizeof(AcaQueue), st);
    if (e == cudaSuccess) {
        AcaWork w{(const AcaJob *)b, (const int64_t *)(b + jb),
                  {(int64_t)cls[0].size(), (int64_t)cls[1].size(), (int64_t)cls[2].size(),
                   (int64_t)cls[3].size(), (int64_t)cls[4].size()},
                  max_big, max_small};
        w.n_jobs = (int64_t)jobs.size();
        // a share of the SMs: 2 CTAs of the ACA fit on an SM
        if (sm_share < 1.0) w.max_ctas = std::max(1, (int)(sm_share * 2 * D.num_sms));
        e = launch_aca(w, D.rule, aop, H0->cplx, H0->prec, Q, D.num_sms, st, 1, H0->has_rules);
    }
    cudaFreeAsync(buf, st);
    CU(e);
    return BEM_OK;
}

}  // namespace bem

extern "C" {

int hmat_build_tree(bem_mesh mesh, int32_t leaf_size, double eta, bem_hmat *out)
{
    return hmat_build_tree_impl(mesh, leaf_size, eta, 0, out, BEM_P0);
}

int hmat_build_tree_space(bem_mesh mesh, int32_t leaf_size, double eta, int32_t space,
                          bem_hmat *out)
{
    return hmat_build_tree_impl(mesh, leaf_size, eta, 0, out, space);
}

int hmat_build_tree_part(bem_mesh mesh, int32_t leaf_size, double eta, int32_t n_parts,
                         int32_t part, bem_hmat *out)
{
    return hmat_build_tree_impl(mesh, leaf_size, eta, 0, out, BEM_P0, n_parts, part);
}

int hmat_part_rows(bem_hmat H, int64_t *row_begin, int64_t *row_end)
{
    if (!H || !row_begin || !row_end) return fail(BEM_E_ARG, "null argument");
    *row_begin = H->row_b * H->dofs;
    *row_end = (H->row_e < 0 ? H->mesh->nt : H->row_e) * H->dofs;
    return BEM_OK;
}

int bem_partition_rows(const int64_t *blocks, int64_t n_blocks, int64_t n_rows, int32_t n_parts,
                       double rank_est, int64_t *bounds)
{
    return guarded([&]() -> int {
        if (!blocks || !bounds || n_blocks < 0 || n_rows < 0 || n_parts < 1 || !(rank_est > 0))
            return fail(BEM_E_ARG, "bad partition arguments");
        for (int64_t b = 0; b < n_blocks; ++b) {
            const int64_t *r = blocks + 5 * b;
            if (r[0] < 0 || r[1] > n_rows || r[0] > r[1] || r[2] > r[3])
                return fail(BEM_E_ARG, "block outside the rows");
        }
        partition_rows(blocks, n_blocks, n_rows, n_parts, rank_est, bounds);
        return BEM_OK;
    });
}

int64_t hmat_dofs(bem_hmat H)
{
    if (!H) return -1;
    return H->space == BEM_P1 ? H->mesh->nv : H->ndof;
}

int hmat_assemble(bem_hmat H, int32_t op, double k, double aca_eps, int32_t prec, void *cuda_stream)
{
    return guarded([&]() -> int {
        cudaStream_t st = (cudaStream_t)cuda_stream;
        int rc = assemble_begin(H, op, k, aca_eps, prec, st);
        if (rc != BEM_OK) return rc;
        bool use_graphs;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            use_graphs = g_tuning.use_graphs != 0;
        }
        // the whole sequence: near field (regular, then singular pairs, FP64),
        // then the persistent ACA over all admissible blocks and its totals
        // the whole sequence: near field (regular, then singular pairs, FP64),
        // then the persistent ACA over all admissible blocks and its totals.
        // (Running the near field on a second stream beside the ACA was
        // measured: the step took as long, the ACA slowing by what the near
        // field saved.)
        auto enqueue = [&](cudaStream_t s, bool capturing) {
            enqueue_near(H, s, capturing);
            enqueue_aca_own(H, s);
            enqueue_finish(H, s, capturing);
        };
        for (int attempt = 0;; ++attempt) {
            assemble_pool(H, st);
            // the first assembly with a given key runs eagerly; the second
            // captures the sequence into a graph, later ones replay it
            const bool same = H->g_op == op && H->g_prec == prec && H->g_k == k &&
                              H->g_eps == aca_eps && H->g_pool == H->d_pool.p &&
                              H->g_near == H->d_near_data.p && H->g_pool_elems == H->pool_elems;
            if (!use_graphs || !same) {
                if (H->graph) {
                    cudaGraphExecDestroy(H->graph);
                    H->graph = nullptr;
                }
                enqueue(st, false);
                H->g_op = op;
                H->g_prec = prec;
                H->g_k = k;
                H->g_eps = aca_eps;
                H->g_pool = H->d_pool.p;
                H->g_near = H->d_near_data.p;
                H->g_pool_elems = H->pool_elems;
            } else {
                if (!H->graph) {
                    // capture on a private stream (the legacy default stream
                    // cannot be captured); the graph is launched on st
                    CU(cudaStreamSynchronize(st));
                    if (!H->cap_stream)
                        CU(cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking));
                    cudaStream_t cs = H->cap_stream;
                    const int64_t before = launches_total();
                    cudaGraph_t gr = nullptr;
                    CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
                    try {
                        enqueue(cs, true);
                    } catch (...) {
                        cudaStreamEndCapture(cs, &gr);
                        if (gr) cudaGraphDestroy(gr);
                        throw;
                    }
                    CU(cudaStreamEndCapture(cs, &gr));
                    cudaError_t ie = cudaGraphInstantiate(&H->graph, gr, 0);
                    cudaGraphDestroy(gr);
                    CU(ie);
                    H->g_nodes = launches_total() - before;
                    count_launches(-H->g_nodes);  // captured, not launched
                }
                CU(cudaGraphLaunch(H->graph, st));
                count_launches(H->g_nodes);
            }
            CU(cudaStreamSynchronize(st));
            if (!H->pin_pool->overflow) break;
            if (attempt >= 6) return fail(BEM_E_OOM, "ACA factor pool keeps overflowing");
            H->pool_want *= 2;
        }
        assemble_end(H, st);
        return BEM_OK;
    });
}

}  // extern "C"

extern "C" {

int hmat_matvec(bem_hmat H, const void *x, void *y, int32_t batch, void *cuda_stream)
{
    return guarded([&]() -> int {
        if (!H) return fail(BEM_E_ARG, "null hmat");
        if (!H->assembled) return fail(BEM_E_STATE, "hmat_matvec before hmat_assemble");
        if (batch < 0) return fail(BEM_E_ARG, "negative batch");
        if (batch == 0) return BEM_OK;
        if (!x || !y) return fail(BEM_E_ARG, "null vector");
        cudaStream_t st = (cudaStream_t)cuda_stream;
        const int64_t nd = H->ndof;
        const bool p1 = H->space == BEM_P1;
        const int64_t nio = p1 ? H->mesh->nv : nd;  // length of the caller's vectors
        const size_t esz = H->cplx ? 16 : 8;
        const size_t vb = nio * esz;
        const bool hx = !is_device_ptr(x), hy = !is_device_ptr(y);
        if ((hx || hy) && H->d_x.bytes < vb) {
            H->d_x.alloc(vb, st);
            H->d_y.alloc(vb, st);
        }
        const int32_t *perm = H->dofs == 1 ? H->d_perm.as<int32_t>() : H->d_dperm.as<int32_t>();
        // the DP1 (or P0) product in the mesh's dof order
        auto apply = [&](const void *xi, void *yo) {
            CU(launch_matvec(H->cplx, nd, perm, xi, yo, H->d_xt.p, H->d_yt.p, H->d_tbuf.p,
                             H->d_far.as<FarBlock>(), H->d_chunks.as<FarChunks>(),
                             (int64_t)H->far.size(), H->d_toff.as<int64_t>(), H->d_pool.p,
                             H->d_near.as<NearBlock>(), H->d_near_data.p,
                             H->d_leaf_rows.as<int64_t>(), H->d_leaf_ptr.as<int64_t>(),
                             H->d_leaf_items.as<int64_t>(), (int64_t)(H->leaf_ptr.size() - 1),
                             H->d_long.as<int64_t>(), (int64_t)H->long_ids.size(),
                             H->d_long_off.as<int64_t>(), st));
        };
        const DevGeom &mg = H->mesh->geom.g;
        for (int32_t b = 0; b < batch; ++b) {
            const void *xb = (const char *)x + b * vb;
            void *yb = (char *)y + b * vb;
            const void *dx = xb;
            void *dy = yb;
            if (hx) {
                CU(cudaMemcpyAsync(H->d_x.p, xb, vb, cudaMemcpyHostToDevice, st));
                dx = H->d_x.p;
            }
            if (hy) dy = H->d_y.p;
            if (!p1) {
                apply(dx, dy);
            } else if (H->op != BEM_HYPS) {
                CU(launch_p1_gather(H->cplx, mg.tri, mg.nt, dx, H->d_xs.p, st));
                apply(H->d_xs.p, H->d_ys.p);
                CU(launch_p1_scatter(H->cplx, H->d_vptr.as<int64_t>(), H->d_vdof.as<int32_t>(),
                                     nio, H->d_ys.p, dy, st));
            } else {
                const int nvec = H->k != 0.0 ? 6 : 3;
                CU(launch_hyps_in(H->cplx, mg, dx, H->d_xs.p, nvec, st));
                for (int j = 0; j < nvec; ++j)
                    apply(H->d_xs.as<char>() + j * nd * esz, H->d_ys.as<char>() + j * nd * esz);
                CU(launch_hyps_out(H->cplx, H->d_vptr.as<int64_t>(), H->d_vdof.as<int32_t>(), mg,
                                   nio, H->k, H->d_ys.p, nvec, dy, st));
            }
            if (hy) CU(cudaMemcpyAsync(yb, dy, vb, cudaMemcpyDeviceToHost, st));
        }
        if (hx || hy) CU(cudaStreamSynchronize(st));
        return BEM_OK;
    });
}

int hmat_stats(bem_hmat H, bem_hmat_stats *out)
{
    return guarded([&]() -> int {
        if (!H || !out) return fail(BEM_E_ARG, "null argument");
        bem_hmat_stats s{};
        s.n_triangles = H->mesh->nt;
        s.n_clusters = (int64_t)H->cl.size();
        s.n_blocks_near = (int64_t)H->near.size();
        s.n_blocks_far = (int64_t)H->far.size();
        for (const FarBlock &F : H->far) {
            s.n_blocks_rule3 += F.rule == kRule3;
            s.n_blocks_rule1 += F.rule == kRule1;
        }
        s.rho3 = H->rho3;
        s.rho1 = H->rho1;
        s.n_blocks_cta = H->nshape[kShapeCta];
        s.n_blocks_warp = H->nshape[kShapeWarp] + H->nshape[kShapeHalf] + H->nshape[kShapeQuarter];
        s.n_blocks_lane = H->nshape[kShapeLane];
        s.n_blocks_half_warp = H->nshape[kShapeHalf];
        s.n_blocks_quarter_warp = H->nshape[kShapeQuarter];
        s.near_entries = H->near_total;
        for (int c = 0; c < 3; ++c) s.singular_pairs[c] = H->sing_entries[c];
        s.far_entries = H->far_entries;
        const size_t esz = H->cplx ? 16 : 8;
        s.factor_bytes = H->factor_elems * (int64_t)esz;
        s.near_bytes = H->near_total * (int64_t)esz;
        s.rank_min = H->rank_min;
        s.rank_max = H->rank_max;
        s.rank_mean = H->far.empty() ? 0.0 : (double)H->rank_sum / H->far.size();
        s.rank_capped_blocks = H->capped;
        s.time_tree_ms = H->t_tree;
        s.time_near_ms = H->t_near;
        s.time_far_ms = H->t_far;
        s.time_near_regular_ms = H->t_near_reg;
        s.time_singular_ms = H->t_near - H->t_near_reg;
        s.aca_fp64_fma = H->k2mn;
        s.assembled = H->assembled;
        s.op = H->op;
        s.k = H->k;
        s.aca_eps = H->eps;
        s.prec = H->prec;
        s.space = H->space;
        s.n_dofs = H->space == BEM_P1 ? H->mesh->nv : H->ndof;
        s.time_tree_clusters_ms = H->t_clusters;
        s.time_tree_blocks_ms = H->t_blocks;
        s.time_tree_lists_ms = H->t_lists;
        s.time_tree_upload_ms = H->t_upload;
        s.factor_read_bytes = H->rank_mn * (int64_t)esz;
        *out = s;
        return BEM_OK;
    });
}

int hmat_blocks(bem_hmat H, int64_t *blocks, int64_t cap, int64_t *n_blocks, int32_t *perm)
{
    return guarded([&]() -> int {
        if (!H || !n_blocks) return fail(BEM_E_ARG, "null argument");
        *n_blocks = (int64_t)H->blocks.size();
        if (perm) std::memcpy(perm, H->perm.data(), H->perm.size() * sizeof(int32_t));
        if (!blocks) return BEM_OK;
        if (cap < (int64_t)H->blocks.size()) return fail(BEM_E_ARG, "block capacity too small");
        for (size_t b = 0; b < H->blocks.size(); ++b) {
            const Cluster &T = H->cl[H->blocks[b].tau], &S = H->cl[H->blocks[b].sigma];
            int64_t *r = blocks + 5 * b;
            r[0] = T.b * H->dofs;
            r[1] = T.e * H->dofs;
            r[2] = S.b * H->dofs;
            r[3] = S.e * H->dofs;
            r[4] = H->blocks[b].adm ? 1 : 0;
        }
        return BEM_OK;
    });
}

int hmat_block_rules(bem_hmat H, int32_t *points, int64_t cap)
{
    return guarded([&]() -> int {
        if (!H || !points) return fail(BEM_E_ARG, "null argument");
        if (cap < (int64_t)H->blocks.size()) return fail(BEM_E_ARG, "capacity too small");
        for (size_t b = 0; b < H->blocks.size(); ++b) points[b] = 0;
        for (size_t f = 0; f < H->far.size(); ++f) {
            const int r = H->far[f].rule;
            points[H->far_block_id[f]] = r == kRule1 ? 1 : (r == kRule3 ? 3 : 6);
        }
        return BEM_OK;
    });
}

int hmat_block_dense(bem_hmat H, int64_t block, void *out, int32_t *rank)
{
    return guarded([&]() -> int {
        if (!H || !out) return fail(BEM_E_ARG, "null argument");
        if (!H->assembled) return fail(BEM_E_STATE, "not assembled");
        if (block < 0 || block >= (int64_t)H->blocks.size()) return fail(BEM_E_ARG, "bad block");
        const size_t esz = H->cplx ? 16 : 8;
        if (!H->blocks[block].adm) {
            auto it = std::find(H->near_block_id.begin(), H->near_block_id.end(), block);
            const NearBlock &N = H->near[it - H->near_block_id.begin()];
            const int64_t m = N.te - N.tb, n = N.se - N.sb;
            std::vector<char> colmajor((size_t)(m * n) * esz);
            CU(cudaMemcpy(colmajor.data(), H->d_near_data.as<char>() + N.off * esz, colmajor.size(),
                          cudaMemcpyDeviceToHost));
            // the device keeps the block column-major; the caller gets rows
            char *o = (char *)out;
            for (int64_t i = 0; i < m; ++i)
                for (int64_t j = 0; j < n; ++j)
                    std::memcpy(o + (i * n + j) * esz, colmajor.data() + (j * m + i) * esz, esz);
            if (rank) *rank = -1;
            return BEM_OK;
        }
        if (!H->far_result_valid) {
            H->far_result.resize(H->far.size());
            CU(cudaMemcpy(H->far_result.data(), H->d_far.p, H->far.size() * sizeof(FarBlock),
                          cudaMemcpyDeviceToHost));
            H->far_result_valid = true;
        }
        auto it = std::find(H->far_block_id.begin(), H->far_block_id.end(), block);
        const int64_t f = it - H->far_block_id.begin();
        const FarBlock &F = H->far_result[f];
        FarChunks C;
        CU(cudaMemcpy(&C, H->d_chunks.as<FarChunks>() + f, sizeof(FarChunks), cudaMemcpyDeviceToHost));
        const int64_t m = F.te - F.tb, n = F.se - F.sb;
        const int r = F.rank;
        if (rank) *rank = r;
        const int cpl = H->cplx ? 2 : 1;
        std::vector<double> U((size_t)m * r * cpl), V((size_t)n * r * cpl);
        for (int l = 0; l < r; ++l) {
            const int64_t base = C.c[l / KCHUNK];
            CU(cudaMemcpy(&U[(size_t)l * m * cpl], H->d_pool.as<char>() + (base + (l % KCHUNK) * m) * esz,
                          m * esz, cudaMemcpyDeviceToHost));
            CU(cudaMemcpy(&V[(size_t)l * n * cpl],
                          H->d_pool.as<char>() + (base + KCHUNK * m + (l % KCHUNK) * n) * esz, n * esz,
                          cudaMemcpyDeviceToHost));
        }
        double *o = (double *)out;
        for (int64_t i = 0; i < m; ++i)
            for (int64_t j = 0; j < n; ++j) {
                double re = 0, im = 0;
                for (int l = 0; l < r; ++l) {
                    if (cpl == 1) {
                        re += U[(size_t)l * m + i] * V[(size_t)l * n + j];
                    } else {
                        double ur = U[2 * ((size_t)l * m + i)], ui = U[2 * ((size_t)l * m + i) + 1];
                        double vr = V[2 * ((size_t)l * n + j)], vi = V[2 * ((size_t)l * n + j) + 1];
                        re += ur * vr - ui * vi;
                        im += ur * vi + ui * vr;
                    }
                }
                if (cpl == 1) o[i * n + j] = re;
                else {
                    o[2 * (i * n + j)] = re;
                    o[2 * (i * n + j) + 1] = im;
                }
            }
        return BEM_OK;
    });
}

int hmat_destroy(bem_hmat H)
{
    return guarded([&]() -> int {
        if (!H) return fail(BEM_E_ARG, "null hmat");
        cudaDeviceSynchronize();  // products on any stream may still read the factors
        --H->mesh->hmat_refs;
        delete H;
        return BEM_OK;
    });
}

}  // extern "C"
