"""ctypes binding of libgs103.so: the C ABI declared in include/gs103.h.

Every function here has the name of the C entry point it calls and only
marshals arguments: torch tensors become device pointers, cameras become a
gs_camera array, the current torch stream becomes the cudaStream_t.  All the
arithmetic runs in the CUDA library.  There is no fallback: if the library is
missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

PKG = Path(__file__).resolve().parent
LIB_PATH = PKG / "_build" / "libgs103.so"

GS_OK, GS_ERR_ARG, GS_ERR_CAPACITY, GS_ERR_CUDA, GS_ERR_TIMEOUT, GS_ERR_NONFINITE = range(6)
GS_F32, GS_BF16, GS_F16 = 0, 1, 2
GS_EW_NONFINITE, GS_EW_CAPACITY, GS_EW_TIMEOUT, GS_EW_BOUNDS = 1, 2, 4, 8
GS_COLOUR_PLANAR_GLOBAL, GS_COLOUR_INTERLEAVED_GLOBAL, GS_COLOUR_PLANAR_STAGED, GS_COLOUR_INTERLEAVED_STAGED = 0, 1, 2, 3
COLOUR_LAYOUTS = {"planar_global": GS_COLOUR_PLANAR_GLOBAL, "interleaved_global": GS_COLOUR_INTERLEAVED_GLOBAL,
                  "planar_staged": GS_COLOUR_PLANAR_STAGED, "interleaved_staged": GS_COLOUR_INTERLEAVED_STAGED}
GS_SCHED_RASTER, GS_SCHED_ORDER = 0, 1
GS_MAX_VIEWS = 64
SPLAT_BYTES = {GS_F32: 48, GS_BF16: 32, GS_F16: 32}

# Every symbol include/gs103.h declares.
EXPORTS = ["gs_version", "gs_strerror", "gs_launch_count", "gs_set_wait_limit", "gs_get_wait_limit", "gs_zero", "gs_project", "gs_colour_records", "gs_colour_repaired", "gs_bin_sort_workspace", "gs_bin_sort", "gs_bin_sort_noalloc",
           "gs_bin_sort_prefix_workspace", "gs_bin_sort_prefix", "gs_bin_sort_prefix_repair",
           "gs_render_fwd", "gs_l1_loss", "gs_render_bwd", "gs_project_bwd", "gs_project_bwd_adam", "gs_adam_step",
           "gs_adam_flat", "gs_tile_features", "gs_mlp_predict", "gs_mlp_grad",
           "gs_mlp_train_step", "gs_rank_judge", "gs_bwd_tile_features", "gs_int_cost", "gs_range_cost", "gs_sched_order_workspace",
           "gs_sched_order", "gs_grad2d_norm", "gs_densify_workspace", "gs_densify",
           "gs_colour_arrays", "gs_render_fwd_colour", "gs_density_workspace", "gs_density_stats",
           "gs_density_control", "gs_colour_buckets", "gs_colour_merge"]


class GsError(RuntimeError):
    pass


class GsCamera(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int), ("H", ctypes.c_int),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3),
                ("campos", ctypes.c_float * 3), ("znear", ctypes.c_float),
                ("bg", ctypes.c_float * 3)]


class GsSchedule(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("d_order", ctypes.c_void_p),
                ("d_queue", ctypes.c_void_p), ("budget_ns", ctypes.c_longlong),
                ("d_n_order", ctypes.c_void_p), ("d_split", ctypes.c_void_p),
                ("d_tile_ns", ctypes.c_void_p), ("d_split_cost", ctypes.c_void_p)]


_lib = None
VP = ctypes.c_void_p
I32 = ctypes.c_int
I64 = ctypes.c_longlong
F32 = ctypes.c_float
SZ = ctypes.c_size_t


def lib():
    """Load the CUDA library (built by paper_2510_14564_gb300.build)."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise GsError(f"CUDA library not built: {LIB_PATH} is missing "
                          "(run python -m paper_2510_14564_gb300.build)")
        L = ctypes.CDLL(str(LIB_PATH))
        P = ctypes.POINTER
        L.gs_version.restype = I32
        L.gs_launch_count.restype = I64
        L.gs_set_wait_limit.argtypes = [I64]
        L.gs_zero.argtypes = [VP, SZ, VP]
        L.gs_get_wait_limit.restype = I64
        L.gs_strerror.restype = ctypes.c_char_p
        L.gs_strerror.argtypes = [I32]
        L.gs_project.argtypes = [P(GsCamera), I32, I32, VP, VP, VP, VP, VP, I32, VP, I32, VP, VP, VP,
                                 VP, VP, VP]
        L.gs_bin_sort_workspace.argtypes = [I32, I32, I64, P(GsCamera), P(SZ)]
        L.gs_bin_sort.argtypes = [P(GsCamera), I32, I32, VP, VP, VP, I64, VP, VP, VP, VP, VP, SZ, VP, VP]
        L.gs_bin_sort_prefix_workspace.argtypes = [I32, I32, I64, P(GsCamera), P(SZ)]
        L.gs_bin_sort_prefix.argtypes = [P(GsCamera), I32, I32, VP, VP, VP, VP, I32, VP, I64, VP, VP, VP, VP,
                                         VP, VP, VP, VP, ctypes.c_uint32, VP, SZ, VP, VP]
        L.gs_colour_records.argtypes = [P(GsCamera), I32, I32, VP, VP, I32, VP, VP, VP, I32, VP]
        L.gs_colour_repaired.argtypes = [P(GsCamera), I32, I32, VP, VP, I32, VP, I64, VP, VP, VP, VP,
                                         ctypes.c_uint32, VP, I32, VP]
        L.gs_bin_sort_prefix_repair.argtypes = [P(GsCamera), I32, I32, VP, VP, VP, VP, I64, VP, VP, VP, VP,
                                                SZ, VP, VP]
        L.gs_bin_sort_noalloc.argtypes = [P(GsCamera), I32, I32, VP, VP, VP, I64, VP, VP, VP, VP, VP, VP]
        L.gs_render_fwd.argtypes = [P(GsCamera), I32, VP, VP, VP, I32, P(GsSchedule), VP, VP, VP, VP,
                                    VP, VP, VP, VP, VP, VP]
        L.gs_l1_loss.argtypes = [I64, VP, VP, VP, VP, VP]
        L.gs_render_bwd.argtypes = [P(GsCamera), I32, VP, VP, VP, I32, P(GsSchedule), VP, VP, VP, VP,
                                    VP, VP, VP]
        L.gs_project_bwd.argtypes = [P(GsCamera), I32, I32, VP, VP, VP, VP, VP, I32, VP, VP, VP, VP]
        L.gs_project_bwd_adam.argtypes = [P(GsCamera), I32, I32, VP, VP, I32, VP, VP, VP, VP, P(F32), F32, F32,
                                          F32, I32, VP, I32, VP, VP]
        L.gs_adam_step.argtypes = [I32, VP, VP, VP, VP, P(F32), F32, F32, F32, I32, VP, I32, VP]
        L.gs_adam_flat.argtypes = [I64, VP, VP, VP, VP, F32, F32, F32, F32, I32, VP]
        L.gs_tile_features.argtypes = [P(GsCamera), I32, VP, VP, VP, I32, I32, VP, VP, VP, VP]
        L.gs_mlp_predict.argtypes = [VP, VP, I32, VP, VP]
        L.gs_bwd_tile_features.argtypes = [P(GsCamera), I32, VP, VP, VP, VP, VP, VP, VP, VP]
        L.gs_mlp_grad.argtypes = [VP, VP, VP, VP, I32, VP, VP, VP]
        L.gs_mlp_train_step.argtypes = [VP, VP, VP, VP, I32, F32, VP, VP, VP, I32, VP, VP, VP]
        L.gs_rank_judge.argtypes = [VP, VP, I32, VP, I32, I32, ctypes.c_uint32, VP, VP]
        L.gs_int_cost.argtypes = [VP, I32, VP, VP]
        L.gs_range_cost.argtypes = [VP, I32, VP, VP]
        L.gs_sched_order_workspace.argtypes = [I32, P(SZ)]
        L.gs_sched_order.argtypes = [VP, I32, VP, VP, SZ, VP]
        L.gs_grad2d_norm.argtypes = [I32, I32, VP, VP, VP]
        L.gs_colour_arrays.argtypes = [I64, VP, VP, VP, VP]
        L.gs_density_workspace.argtypes = [I32, P(SZ)]
        L.gs_colour_buckets.argtypes = [I32, VP, VP, VP, I32, VP, VP, VP, VP]
        L.gs_colour_merge.argtypes = [I32, VP, VP, VP, I32, VP, VP, VP, VP, VP, VP]
        L.gs_density_stats.argtypes = [I32, VP, F32, I32, VP, VP, VP, VP, P(F32), VP, VP, SZ, VP]
        L.gs_density_control.argtypes = [I32, VP, VP, VP, VP, VP, F32, I32, F32, F32, F32, F32, F32, I64, VP, VP,
                                         VP, VP, I32, VP, VP, VP, SZ, VP, VP]
        L.gs_render_fwd_colour.argtypes = [P(GsCamera), I32, I32, VP, VP, VP, I32, VP, VP, VP, VP, VP]
        L.gs_densify_workspace.argtypes = [I32, P(SZ)]
        L.gs_densify.argtypes = [I32, VP, VP, VP, VP, F32, I32, I64, VP, VP, VP, VP, I32, VP, VP, SZ, VP, VP]
        for name in EXPORTS:
            if name not in ("gs_version", "gs_strerror", "gs_launch_count", "gs_get_wait_limit"):
                getattr(L, name).restype = I32
        _lib = L
    return _lib


def check(rc: int, what: str) -> None:
    if rc != GS_OK:
        msg = lib().gs_strerror(int(rc)).decode()
        raise GsError(f"{what}: {msg} (status {rc})")


def ptr(t) -> int | None:
    """Device pointer of a tensor (None for None)."""
    if t is None:
        return None
    return t.data_ptr()


def stream_ptr(stream=None) -> int | None:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream or None


def camera_array(cams) -> ctypes.Array:
    """gs_camera[] from scenes.Camera objects (host memory)."""
    if len(cams) < 1 or len(cams) > GS_MAX_VIEWS:
        raise GsError(f"need 1..{GS_MAX_VIEWS} views, got {len(cams)}")
    arr = (GsCamera * len(cams))()
    for c, cam in zip(arr, cams):
        c.W, c.H = int(cam.W), int(cam.H)
        c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
        for k, v in enumerate(np.asarray(cam.R, np.float32).ravel()):
            c.R[k] = float(v)
        for k, v in enumerate(np.asarray(cam.t, np.float32).ravel()):
            c.t[k] = float(v)
        for k, v in enumerate(np.asarray(cam.campos, np.float32).ravel()):
            c.campos[k] = float(v)
        c.znear = float(cam.znear)
        for k, v in enumerate(cam.bg):
            c.bg[k] = float(v)
    return arr


# ---------------------------------------------------------------------------
# Entry points (argument marshalling only)
# ---------------------------------------------------------------------------

def gs_version() -> int:
    return int(lib().gs_version())


def gs_strerror(status: int) -> str:
    return lib().gs_strerror(int(status)).decode()


def gs_launch_count() -> int:
    return int(lib().gs_launch_count())


def gs_zero(t, stream=None) -> None:
    """Zero a tensor's bytes on the stream (cudaMemsetAsync in the library)."""
    check(lib().gs_zero(ptr(t), t.numel() * t.element_size(), stream_ptr(stream)), "gs_zero")


def gs_set_wait_limit(reads: int) -> None:
    check(lib().gs_set_wait_limit(int(reads)), "gs_set_wait_limit")


def gs_get_wait_limit() -> int:
    return int(lib().gs_get_wait_limit())


def gs_project(cams, N, means, log_scales, quats, opacity_logits, sh, sh_dtype, splats, rgb_dtype,
               depth, rect, touched, radius, err_word, stream=None):
    ca = camera_array(cams)
    check(lib().gs_project(ca, len(cams), int(N), ptr(means), ptr(log_scales), ptr(quats),
                           ptr(opacity_logits), ptr(sh), int(sh_dtype), ptr(splats), int(rgb_dtype),
                           ptr(depth), ptr(rect), ptr(touched), ptr(radius), ptr(err_word),
                           stream_ptr(stream)), "gs_project")


def gs_bin_sort_workspace(cams, N, capacity) -> int:
    ca = camera_array(cams)
    out = SZ(0)
    check(lib().gs_bin_sort_workspace(len(cams), int(N), int(capacity), ca, ctypes.byref(out)),
          "gs_bin_sort_workspace")
    return int(out.value)


def gs_bin_sort(cams, N, depth, rect, touched, capacity, vals, tile_ranges, keys, n_instances,
                workspace, err_word, stream=None):
    ca = camera_array(cams)
    check(lib().gs_bin_sort(ca, len(cams), int(N), ptr(depth), ptr(rect), ptr(touched),
                            int(capacity), ptr(vals), ptr(tile_ranges), ptr(keys), ptr(n_instances),
                            ptr(workspace), workspace.numel() * workspace.element_size(),
                            ptr(err_word), stream_ptr(stream)), "gs_bin_sort")


def gs_bin_sort_prefix_workspace(cams, N, capacity) -> int:
    ca = camera_array(cams)
    out = SZ(0)
    check(lib().gs_bin_sort_prefix_workspace(len(cams), int(N), int(capacity), ca, ctypes.byref(out)),
          "gs_bin_sort_prefix_workspace")
    return int(out.value)


def gs_bin_sort_prefix(cams, N, depth, rect, touched, splats, rgb_dtype, tile_limit, capacity, vals,
                       tile_ranges, tile_count, keys, n_instances, workspace, err_word, stream=None,
                       colour_list=None, colour_count=None, colour_mark=None, colour_epoch=0):
    ca = camera_array(cams)
    check(lib().gs_bin_sort_prefix(ca, len(cams), int(N), ptr(depth), ptr(rect), ptr(touched), ptr(splats),
                                   int(rgb_dtype), ptr(tile_limit), int(capacity), ptr(vals),
                                   ptr(tile_ranges), ptr(tile_count), ptr(keys), ptr(n_instances),
                                   ptr(colour_list), ptr(colour_count), ptr(colour_mark), int(colour_epoch),
                                   ptr(workspace), workspace.numel() * workspace.element_size(),
                                   ptr(err_word), stream_ptr(stream)), "gs_bin_sort_prefix")


def gs_colour_records(cams, N, means, sh, sh_dtype, rec_list, count, splats, rgb_dtype, stream=None):
    ca = camera_array(cams)
    check(lib().gs_colour_records(ca, len(cams), int(N), ptr(means), ptr(sh), int(sh_dtype), ptr(rec_list),
                                  ptr(count), ptr(splats), int(rgb_dtype), stream_ptr(stream)),
          "gs_colour_records")


def gs_colour_repaired(cams, N, means, sh, sh_dtype, vals, capacity, tiles, n_tiles, tile_ranges, mark, epoch,
                       splats, rgb_dtype, stream=None):
    ca = camera_array(cams)
    check(lib().gs_colour_repaired(ca, len(cams), int(N), ptr(means), ptr(sh), int(sh_dtype), ptr(vals),
                                   int(capacity), ptr(tiles), ptr(n_tiles), ptr(tile_ranges), ptr(mark),
                                   int(epoch), ptr(splats), int(rgb_dtype), stream_ptr(stream)),
          "gs_colour_repaired")


def gs_bin_sort_prefix_repair(cams, N, rect, touched, flag_tiles, flag_count, capacity, vals,
                              tile_ranges, n_instances, workspace, err_word, stream=None):
    ca = camera_array(cams)
    check(lib().gs_bin_sort_prefix_repair(ca, len(cams), int(N), ptr(rect), ptr(touched), ptr(flag_tiles),
                                          ptr(flag_count), int(capacity), ptr(vals), ptr(tile_ranges),
                                          ptr(n_instances), ptr(workspace),
                                          workspace.numel() * workspace.element_size(), ptr(err_word),
                                          stream_ptr(stream)), "gs_bin_sort_prefix_repair")


def gs_bin_sort_noalloc(cams, N, depth, rect, touched, capacity, vals, tile_ranges, keys, n_instances,
                        err_word, stream=None):
    ca = camera_array(cams)
    check(lib().gs_bin_sort_noalloc(ca, len(cams), int(N), ptr(depth), ptr(rect), ptr(touched),
                                    int(capacity), ptr(vals), ptr(tile_ranges), ptr(keys),
                                    ptr(n_instances), ptr(err_word), stream_ptr(stream)),
          "gs_bin_sort_noalloc")


def _sched(sched):
    if sched is None:
        return None
    s = GsSchedule()
    s.mode = int(sched.get("mode", GS_SCHED_RASTER))
    s.d_order = ptr(sched.get("order"))
    s.d_queue = ptr(sched.get("queue"))
    s.budget_ns = int(sched.get("budget_ns", 0))
    s.d_n_order = ptr(sched.get("n_order"))
    s.d_split = ptr(sched.get("split"))
    s.d_tile_ns = ptr(sched.get("tile_ns"))
    s.d_split_cost = ptr(sched.get("split_cost"))
    return ctypes.byref(s), s


def gs_render_fwd(cams, tile_ranges, vals, splats, rgb_dtype, sched, img, T_final, n_proc,
                  tile_nproc, tile_ns, err_word, stream=None, tile_count=None, flag_tiles=None,
                  flag_count=None):
    ca = camera_array(cams)
    sp = _sched(sched)
    check(lib().gs_render_fwd(ca, len(cams), ptr(tile_ranges), ptr(vals), ptr(splats), int(rgb_dtype),
                              sp[0] if sp else None, ptr(img), ptr(T_final), ptr(n_proc),
                              ptr(tile_nproc), ptr(tile_ns), ptr(tile_count), ptr(flag_tiles),
                              ptr(flag_count), ptr(err_word), stream_ptr(stream)), "gs_render_fwd")


def gs_l1_loss(n, img, tgt, loss, dimg, stream=None):
    check(lib().gs_l1_loss(int(n), ptr(img), ptr(tgt), ptr(loss), ptr(dimg), stream_ptr(stream)),
          "gs_l1_loss")


def gs_render_bwd(cams, tile_ranges, vals, splats, rgb_dtype, sched, dimg, T_final, n_proc,
                  tile_nproc, grad2d, err_word, stream=None):
    ca = camera_array(cams)
    sp = _sched(sched)
    check(lib().gs_render_bwd(ca, len(cams), ptr(tile_ranges), ptr(vals), ptr(splats), int(rgb_dtype),
                              sp[0] if sp else None, ptr(dimg), ptr(T_final), ptr(n_proc),
                              ptr(tile_nproc), ptr(grad2d), ptr(err_word), stream_ptr(stream)),
          "gs_render_bwd")


def gs_project_bwd(cams, N, means, log_scales, quats, opacity_logits, sh, sh_dtype, touched, grad2d,
                   dparams, stream=None):
    ca = camera_array(cams)
    check(lib().gs_project_bwd(ca, len(cams), int(N), ptr(means), ptr(log_scales), ptr(quats),
                               ptr(opacity_logits), ptr(sh), int(sh_dtype), ptr(touched), ptr(grad2d),
                               ptr(dparams), stream_ptr(stream)), "gs_project_bwd")


def gs_project_bwd_adam(cams, N, params, sh, sh_dtype, touched, grad2d, m, v, lr6, b1, b2, eps, t,
                        sh_shadow=None, shadow_dtype=GS_BF16, dparams=None, stream=None):
    ca = camera_array(cams)
    lr = (F32 * 6)(*[float(x) for x in lr6])
    check(lib().gs_project_bwd_adam(ca, len(cams), int(N), ptr(params), ptr(sh), int(sh_dtype), ptr(touched),
                                    ptr(grad2d), ptr(m), ptr(v), lr, float(b1), float(b2), float(eps), int(t),
                                    ptr(sh_shadow), int(shadow_dtype), ptr(dparams), stream_ptr(stream)),
          "gs_project_bwd_adam")


def gs_adam_step(N, params, grads, m, v, lr6, b1, b2, eps, t, sh_shadow=None, shadow_dtype=GS_BF16,
                 stream=None):
    lr = (F32 * 6)(*[float(x) for x in lr6])
    check(lib().gs_adam_step(int(N), ptr(params), ptr(grads), ptr(m), ptr(v), lr, float(b1), float(b2),
                             float(eps), int(t), ptr(sh_shadow), int(shadow_dtype), stream_ptr(stream)),
          "gs_adam_step")


def gs_adam_flat(n, p, g, m, v, lr, b1, b2, eps, t, stream=None):
    check(lib().gs_adam_flat(int(n), ptr(p), ptr(g), ptr(m), ptr(v), float(lr), float(b1), float(b2),
                             float(eps), int(t), stream_ptr(stream)), "gs_adam_flat")


def gs_grad2d_norm(n_views, N, grad2d, out, stream=None):
    check(lib().gs_grad2d_norm(int(n_views), int(N), ptr(grad2d), ptr(out), stream_ptr(stream)),
          "gs_grad2d_norm")


def gs_densify_workspace(N) -> int:
    out = SZ(0)
    check(lib().gs_densify_workspace(int(N), ctypes.byref(out)), "gs_densify_workspace")
    return int(out.value)


def gs_densify(N, params, m, v, grad_norm, logit_threshold, n_clone, capacity, params_out, m_out, v_out,
               sh_shadow_out, shadow_dtype, n_out, workspace, err_word, stream=None):
    check(lib().gs_densify(int(N), ptr(params), ptr(m), ptr(v), ptr(grad_norm), float(logit_threshold),
                           int(n_clone), int(capacity), ptr(params_out), ptr(m_out), ptr(v_out),
                           ptr(sh_shadow_out), int(shadow_dtype), ptr(n_out), ptr(workspace),
                           workspace.numel() * workspace.element_size(), ptr(err_word), stream_ptr(stream)),
          "gs_densify")


def gs_colour_arrays(VN, splats, planar, interleaved, stream=None):
    check(lib().gs_colour_arrays(int(VN), ptr(splats), ptr(planar), ptr(interleaved), stream_ptr(stream)),
          "gs_colour_arrays")


def gs_render_fwd_colour(cams, N, tile_ranges, vals, splats, layout, colour, img, T_final, n_proc, stream=None):
    ca = camera_array(cams)
    check(lib().gs_render_fwd_colour(ca, len(cams), int(N), ptr(tile_ranges), ptr(vals), ptr(splats), int(layout),
                                     ptr(colour), ptr(img), ptr(T_final), ptr(n_proc), stream_ptr(stream)),
          "gs_render_fwd_colour")


def gs_density_workspace(N) -> int:
    out = SZ(0)
    check(lib().gs_density_workspace(int(N), ctypes.byref(out)), "gs_density_workspace")
    return int(out.value)


def gs_density_stats(N, means, r, k, rho, dbar, nn, dnn, thr_params=None, thresholds=None, workspace=None,
                     stream=None):
    tp = (F32 * 3)(*[float(x) for x in thr_params]) if thr_params is not None else None
    check(lib().gs_density_stats(int(N), ptr(means), float(r), int(k), ptr(rho), ptr(dbar), ptr(nn), ptr(dnn), tp,
                                 ptr(thresholds), ptr(workspace),
                                 workspace.numel() * workspace.element_size() if workspace is not None else 0,
                                 stream_ptr(stream)), "gs_density_stats")


def gs_density_control(N, params, m, v, z, u, r, k, alpha, beta, alpha_d, delta, gamma, capacity, params_out,
                       m_out, v_out, sh_shadow_out, shadow_dtype, n_out, thresholds, workspace, err_word,
                       stream=None):
    check(lib().gs_density_control(int(N), ptr(params), ptr(m), ptr(v), ptr(z), ptr(u), float(r), int(k),
                                   float(alpha), float(beta), float(alpha_d), float(delta), float(gamma),
                                   int(capacity), ptr(params_out), ptr(m_out), ptr(v_out), ptr(sh_shadow_out),
                                   int(shadow_dtype), ptr(n_out), ptr(thresholds), ptr(workspace),
                                   workspace.numel() * workspace.element_size(), ptr(err_word),
                                   stream_ptr(stream)), "gs_density_control")


def gs_colour_buckets(n_tiles, tile_ranges, vals, splats, rgb_dtype, count, sums, tile_distinct, stream=None):
    check(lib().gs_colour_buckets(int(n_tiles), ptr(tile_ranges), ptr(vals), ptr(splats), int(rgb_dtype), ptr(count),
                                  ptr(sums), ptr(tile_distinct), stream_ptr(stream)), "gs_colour_buckets")


def gs_colour_merge(n_tiles, tile_ranges, vals, splats, rgb_dtype, out_ranges, out_vals, out_splats,
                    out_src=None, out_members=None, stream=None):
    check(lib().gs_colour_merge(int(n_tiles), ptr(tile_ranges), ptr(vals), ptr(splats), int(rgb_dtype),
                                ptr(out_ranges), ptr(out_vals), ptr(out_splats), ptr(out_src), ptr(out_members),
                                stream_ptr(stream)), "gs_colour_merge")


def gs_tile_features(cams, tile_ranges, vals, splats, rgb_dtype, cap, feats, w16=None, pred=None,
                     stream=None):
    ca = camera_array(cams)
    check(lib().gs_tile_features(ca, len(cams), ptr(tile_ranges), ptr(vals), ptr(splats),
                                 int(rgb_dtype), int(cap), ptr(feats), ptr(w16), ptr(pred),
                                 stream_ptr(stream)), "gs_tile_features")


def gs_bwd_tile_features(cams, tile_ranges, tile_nproc, n_proc, tile_ns, feats, w16=None, pred=None, stream=None):
    ca = camera_array(cams)
    check(lib().gs_bwd_tile_features(ca, len(cams), ptr(tile_ranges), ptr(tile_nproc), ptr(n_proc), ptr(tile_ns),
                                     ptr(feats), ptr(w16), ptr(pred), stream_ptr(stream)), "gs_bwd_tile_features")


def gs_mlp_predict(w16, feats, n, pred, stream=None):
    check(lib().gs_mlp_predict(ptr(w16), ptr(feats), int(n), ptr(pred), stream_ptr(stream)),
          "gs_mlp_predict")


def gs_mlp_grad(w32, feats, tile_ns, target, n, grad, loss, stream=None):
    check(lib().gs_mlp_grad(ptr(w32), ptr(feats), ptr(tile_ns), ptr(target), int(n), ptr(grad),
                            ptr(loss), stream_ptr(stream)), "gs_mlp_grad")


def gs_mlp_train_step(w32, w16, m, v, t, lr, feats, tile_ns, target, n, grad, loss, stream=None):
    check(lib().gs_mlp_train_step(ptr(w32), ptr(w16), ptr(m), ptr(v), int(t), float(lr), ptr(feats),
                                  ptr(tile_ns), ptr(target), int(n), ptr(grad), ptr(loss),
                                  stream_ptr(stream)), "gs_mlp_train_step")


def gs_rank_judge(a, b, b_stride, tile_ns, n, n_pairs, seed, out, stream=None):
    check(lib().gs_rank_judge(ptr(a), ptr(b), int(b_stride), ptr(tile_ns), int(n), int(n_pairs),
                              int(seed) & 0xFFFFFFFF, ptr(out), stream_ptr(stream)), "gs_rank_judge")


def gs_int_cost(counts, n, cost, stream=None):
    check(lib().gs_int_cost(ptr(counts), int(n), ptr(cost), stream_ptr(stream)), "gs_int_cost")


def gs_range_cost(tile_ranges, T, cost, stream=None):
    check(lib().gs_range_cost(ptr(tile_ranges), int(T), ptr(cost), stream_ptr(stream)), "gs_range_cost")


def gs_sched_order_workspace(n) -> int:
    out = SZ(0)
    check(lib().gs_sched_order_workspace(int(n), ctypes.byref(out)), "gs_sched_order_workspace")
    return int(out.value)


def gs_sched_order(cost, n, order, workspace, stream=None):
    check(lib().gs_sched_order(ptr(cost), int(n), ptr(order), ptr(workspace),
                               workspace.numel() * workspace.element_size(), stream_ptr(stream)),
          "gs_sched_order")
