// libins: eddy-viscosity closures (Smagorinsky, WALE, QR, Vreman; ins_set_eddy_viscosity and
// ins_eddy_viscosity in include/ins.h): nu_t at the cell centres and the stress divergence on the faces.
#include "ins_internal.cuh"

namespace {
dim3 eddy_grid(const ins_grid* g) { return dim3((g->nx + 31) / 32, (g->ny + 7) / 8, g->nz); }

template <typename T>
EddyCoef<T> eddy_coef(const ins_grid* g) {
    EddyCoef<T> c;
    c.nx = g->nx;
    c.ny = g->ny;
    c.nz = g->nz;
    double vol = 1.0;
    for (int a = 0; a < 3; ++a) {
        const double d = g->d[a][0];
        c.id[a] = (T)(1.0 / d);
        c.w2[a] = (T)(d * d);
        vol *= d;
    }
    const double D = std::cbrt(vol);
    c.CD2 = (T)((g->eddy_C * D) * (g->eddy_C * D));
    c.C2 = (T)(g->eddy == EDDY_CONSTANT ? g->eddy_C : g->eddy_C * g->eddy_C);
    const T* rows = reinterpret_cast<const T*>(g->eddy_rows);
    c.idy = rows;
    c.ihy = rows ? rows + g->ny : nullptr;
    c.cd2y = rows ? rows + 2 * g->ny : nullptr;
    c.w2y = rows ? rows + 3 * g->ny : nullptr;
    return c;
}

// The per-row wall-normal coefficients of the attached model, in the field type.
template <typename T>
cudaError_t eddy_upload_rows(ins_grid* g) {
    const int ny = g->ny;
    std::vector<T> v(4 * (size_t)ny);
    for (int j = 0; j < ny; ++j) {
        const double dy = g->d[1][j];
        const double D = std::cbrt(g->d[0][0] * dy * g->d[2][0]);
        v[j] = (T)(1.0 / dy);
        v[ny + j] = (T)(1.0 / g->h[1][j]);
        v[2 * ny + j] = (T)((g->eddy_C * D) * (g->eddy_C * D));
        v[3 * ny + j] = (T)(dy * dy);
    }
    return cudaMemcpy(g->eddy_rows, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

template <typename T, bool WALL>
ins_status eddy_nut_launch(ins_grid* g, const T* u, T* nut) {
    const EddyCoef<T> c = eddy_coef<T>(g);
    const dim3 grd = eddy_grid(g), blk(32, 8);
    switch (g->eddy) {
        case EDDY_SMAGORINSKY:
            KLAUNCH(g, "eddy_nut", (k_eddy_nut<T, EDDY_SMAGORINSKY, WALL><<<grd, blk, 0, g->stream>>>(c, u, nut)));
            break;
        case EDDY_WALE: KLAUNCH(g, "eddy_nut", (k_eddy_nut<T, EDDY_WALE, WALL><<<grd, blk, 0, g->stream>>>(c, u, nut))); break;
        case EDDY_QR: KLAUNCH(g, "eddy_nut", (k_eddy_nut<T, EDDY_QR, WALL><<<grd, blk, 0, g->stream>>>(c, u, nut))); break;
        case EDDY_VREMAN:
            KLAUNCH(g, "eddy_nut", (k_eddy_nut<T, EDDY_VREMAN, WALL><<<grd, blk, 0, g->stream>>>(c, u, nut)));
            break;
        default:
            KLAUNCH(g, "eddy_nut", (k_eddy_nut<T, EDDY_CONSTANT, WALL><<<grd, blk, 0, g->stream>>>(c, u, nut)));
            break;
    }
    return INS_OK;
}

}  // namespace

template <typename T>
ins_status eddy_nut(ins_grid* g, const T* u, T* nut) {
    if (g->wall_y) return eddy_nut_launch<T, true>(g, u, nut);
    return eddy_nut_launch<T, false>(g, u, nut);
}

// nu_t into the grid's eddy buffer, then the stress divergence into `term`.
template <typename T>
ins_status eddy_term(ins_grid* g, const T* u, T* term) {
    T* nut = reinterpret_cast<T*>(g->eddy_buf);
    ins_status s = eddy_nut<T>(g, u, nut);
    if (s != INS_OK) return s;
    if (g->wall_y)
        KLAUNCH(g, "eddy_div",
                (k_eddy_div<T, true><<<eddy_grid(g), dim3(32, 8), 0, g->stream>>>(eddy_coef<T>(g), u, nut, term)));
    else
        KLAUNCH(g, "eddy_div",
                (k_eddy_div<T, false><<<eddy_grid(g), dim3(32, 8), 0, g->stream>>>(eddy_coef<T>(g), u, nut, term)));
    return INS_OK;
}

template ins_status eddy_nut<float>(ins_grid*, const float*, float*);
template ins_status eddy_nut<double>(ins_grid*, const double*, double*);
template ins_status eddy_term<float>(ins_grid*, const float*, float*);
template ins_status eddy_term<double>(ins_grid*, const double*, double*);

extern "C" {

ins_status ins_set_eddy_viscosity(ins_grid* g, int model, double C) {
    g_err.clear();
    if (!g) return fail(INS_ERR_ARG, "null grid");
    if (model < INS_EDDY_NONE || model > INS_EDDY_CONSTANT) return fail(INS_ERR_ARG, "unknown eddy-viscosity model");
    if (model == INS_EDDY_NONE) {
        g->eddy = 0;
        return INS_OK;
    }
    if (!(std::isfinite(C) && C >= 0.0)) return fail(INS_ERR_ARG, "C must be finite and >= 0");
    if (g->dim != 3) return fail(INS_ERR_UNSUPPORTED, "eddy-viscosity models: 3-D grids only");
    if (g->nx < 2 || g->ny < 2 || g->nz < 2) return fail(INS_ERR_UNSUPPORTED, "eddy-viscosity models need n >= 2");
    if (g->closure) return fail(INS_ERR_UNSUPPORTED, "a CNN closure is attached (one closure at a time)");
    if (!g->eddy_buf) {
        const size_t bytes = (size_t)4 * g->N * (g->dtype == INS_F64 ? 8 : 4);
        cudaError_t e = cudaMalloc(&g->eddy_buf, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            g->eddy_buf = nullptr;
            return fail(INS_ERR_OOM, "eddy-viscosity buffers");
        }
    }
    if (g->wall_y) {
        if (!g->eddy_rows) {
            cudaError_t e = cudaMalloc(&g->eddy_rows, (size_t)4 * g->ny * (g->dtype == INS_F64 ? 8 : 4));
            if (e != cudaSuccess) {
                cudaGetLastError();
                g->eddy_rows = nullptr;
                return fail(INS_ERR_OOM, "eddy-viscosity row coefficients");
            }
        }
        g->eddy_C = C;
        cudaError_t e = g->dtype == INS_F64 ? eddy_upload_rows<double>(g) : eddy_upload_rows<float>(g);
        if (e != cudaSuccess) return fail(INS_ERR_CUDA, cudaGetErrorString(e));
    }
    g->eddy = model;
    g->eddy_C = C;
    return INS_OK;
}

ins_status ins_eddy_viscosity(ins_grid* g, const void* u, void* nut) {
    g_err.clear();
    if (!g) return fail(INS_ERR_ARG, "null grid");
    CHECK(check_ptr(g, u, "u"));
    if (!nut) return fail(INS_ERR_ARG, "nut is null");
    if (!g->eddy) return fail(INS_ERR_ARG, "no eddy-viscosity model attached");
    if (g->dtype == INS_F64) return eddy_nut<double>(g, (const double*)u, (double*)nut);
    return eddy_nut<float>(g, (const float*)u, (float*)nut);
}

}  // extern "C"
