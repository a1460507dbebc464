"""The C ABI without a GPU: libnif.so loads, exports every function that
include/nif.h declares, its structs have the layout a C compiler gives them,
and host-side argument checks return their status codes."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nif.h")


@pytest.fixture(scope="module")
def L():
    from paper_2306_07191_gb300 import build
    build.build()
    from paper_2306_07191_gb300 import _lib
    return _lib


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+char\s*\*|nif_status|size_t|int64_t|int32_t)\s+(\w+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_every_declared_function_is_exported_and_bound(L):
    names = _declared_functions()
    assert len(names) >= 25
    for n in names:
        assert hasattr(L.lib, n), n
        assert n in L.SIGNATURES, n


def test_struct_layout_matches_the_c_compiler(L):
    fields_m = [f[0] for f in L.ModelDesc._fields_]
    fields_o = [f[0] for f in L.OptimDesc._fields_]
    prog = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){",
            'printf("%zu %zu %zu\\n", sizeof(nif_ray), sizeof(nif_model_desc), sizeof(nif_optim_desc));']
    for f in fields_m:
        prog.append(f'printf("m {f} %zu\\n", offsetof(nif_model_desc, {f}));')
    for f in fields_o:
        prog.append(f'printf("o {f} %zu\\n", offsetof(nif_optim_desc, {f}));')
    prog.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write("\n".join(prog))
        subprocess.check_call(["gcc", "-std=c11", c, "-o", exe])
        out = subprocess.check_output([exe], text=True).split("\n")
    sizes = [int(x) for x in out[0].split()]
    assert sizes == [32, ctypes.sizeof(L.ModelDesc), ctypes.sizeof(L.OptimDesc)]
    for line in out[1:]:
        if not line:
            continue
        kind, name, off = line.split()
        S = L.ModelDesc if kind == "m" else L.OptimDesc
        assert getattr(S, name).offset == int(off), name


def test_host_side_argument_errors(L):
    d = L.ModelDesc()
    assert L.lib.nif_encode(ctypes.byref(d), None, None, None, 0, None, 0, None) == L.NIF_ERR_ARG
    assert "n_features" in L.last_error()
    assert L.lib.bvh_build(None, 0, None, -1, None, None, 0, None, 0, None) == L.NIF_ERR_ARG
    assert L.lib.bvh_cast_shadow(None, None, -5, None, None) == L.NIF_ERR_ARG
    assert L.lib.bvh_cast_shadow(None, None, 0, None, None) == L.NIF_OK  # n == 0 queues nothing
    assert L.lib.nif_adam(None, None, None, None, 10, 1e-2, 0.9, 0.999, 1e-15, 1.0, 0, None, 0, None) == L.NIF_ERR_ARG
    assert L.lib.nif_loss(None, None, 5, 1.0, None, None, None) == L.NIF_ERR_ARG
    assert L.lib.nif_fill_uniform(None, -1, 0, 1.0, None) == L.NIF_ERR_ARG


def _room_desc(L, **kw):
    from paper_2306_07191_gb300 import workloads
    d = L.ModelDesc()
    d.n_levels = 16
    d.n_features = 2
    d.log2_table = 19
    for i, r in enumerate(workloads.ROOM_RES):
        d.res[i] = r
    d.grid_dtype = L.NIF_F16
    d.n_objects = 64
    d.d_obj_aabb = d.d_grids = d.d_weights = 256  # never dereferenced on the host
    d.n_hidden, d.width, d.act = 3, 64, L.NIF_ACT_RELU
    d.mlp_dtype = L.NIF_F16
    d.net_mode, d.n_nets = L.NIF_NETS_CLASS, 2
    for k, v in kw.items():
        setattr(d, k, v)
    return d


def test_sizes_agree_with_the_oracle_layout(L):
    from oracle import nif as onif
    from paper_2306_07191_gb300 import workloads
    d = _room_desc(L)
    sizes, hashed, off = onif.level_layout(workloads.ROOM_RES, 19)
    assert L.lib.nif_grid_vertices(ctypes.byref(d)) == int(off[-1]) == 5723320
    assert sum(hashed) == 10
    assert L.lib.nif_weight_count(ctypes.byref(d)) == 96 * 64 + 2 * 64 * 64 + 64
    assert L.lib.nif_workspace_size(ctypes.byref(d), 1000, 5000) > 2 * 5000 * 4
    assert L.lib.nif_train_workspace_size(ctypes.byref(d), 1000) >= (96 + 3 * 64 + 96 + 2) * 1000 * 4
    bad = _room_desc(L, n_nets=3)
    assert L.lib.nif_workspace_size(ctypes.byref(bad), 1, 1) == 0
    assert L.lib.bvh_build_size(0) > 0 and L.lib.bvh_build_size(1000) >= 1000 * 48


def test_splitmix_generator_matches_hand_values():
    """SplitMix64 (Steele, Lea & Flood 2014) first output for state 0 after one
    increment is 0xE220A8397B1DCDAF; top 24 bits -> u -> 2u - 1."""
    from paper_2306_07191_gb300 import synth
    v = synth.splitmix_uniform(np.array([0]), 0, 1.0)[0]
    top = 0xE220A8397B1DCDAF >> 40
    assert v == np.float32(2.0 * top / 2 ** 24 - 1.0)


def test_spherical_descriptor_sizes(L):
    """nif_grid_vertices / nif_weight_count of the paper's encoding: per
    object [position R*R*N | direction R*R*N | distance R1*N1], K = 2N or
    2N + N1 (the weight counts of Sec. 5's 18 kB / 21 kB networks)."""
    d = _room_desc(L)
    d.n_levels, d.res[0], d.n_features = 1, 256, 3
    d.encoding, d.n_hidden, d.width = L.NIF_ENC_SPHERICAL_OUTER, 2, 64
    assert L.lib.nif_grid_vertices(ctypes.byref(d)) == 2 * 256 * 256 * 3
    assert L.lib.nif_weight_count(ctypes.byref(d)) == 6 * 64 + 64 * 64 + 64
    d.encoding, d.res[0], d.n_features, d.res_1d, d.n_features_1d = L.NIF_ENC_SPHERICAL_INNER, 128, 5, 128, 3
    d.n_hidden, d.width = 3, 48
    assert L.lib.nif_grid_vertices(ctypes.byref(d)) == 2 * 128 * 128 * 5 + 128 * 3
    assert L.lib.nif_weight_count(ctypes.byref(d)) == 13 * 48 + 2 * 48 * 48 + 48
    d.res_1d = 1  # a 1D grid needs two cells
    assert L.lib.nif_grid_vertices(ctypes.byref(d)) == -1


def test_state_checkpoint_size_and_header_checks(L):
    """nif_state_size follows the documented layout; nif_state_load refuses a
    buffer whose header does not match the model (before any device work)."""
    import numpy as np
    d = _room_desc(L)
    P = 96 * 64 + 2 * 64 * 64 + 64
    V = 5723320
    nw, ng = 2 * P, 64 * 2 * V * 2
    size = L.lib.nif_state_size(ctypes.byref(d))
    assert size == 16 * 8 + 4 * 3 * (nw + ng)
    o = L.OptimDesc()
    for name in ("d_w_master", "d_w_grad", "d_w_m", "d_w_v", "d_g_master", "d_g_grad", "d_g_m", "d_g_v"):
        setattr(o, name, 256)  # never dereferenced: the header check fails first
    buf = np.zeros(64, dtype=np.int64)
    assert L.lib.nif_state_load(ctypes.byref(d), ctypes.byref(o), buf.ctypes.data_as(ctypes.c_void_p), size,
                                None) == L.NIF_ERR_ARG
    assert "header word 0" in L.last_error()
    assert L.lib.nif_state_load(ctypes.byref(d), ctypes.byref(o), buf.ctypes.data_as(ctypes.c_void_p), 16,
                                None) == L.NIF_ERR_ARG
    # the same array sizes saved from a model with another encoding, network
    # mode, output count, level count, feature count, grid dtype or level
    # layout: refused at that header word
    good = [0x5346494E, 2, 96, 64, 3, 2, nw, ng, 7, L.NIF_ENC_MULTIRES, L.NIF_NETS_CLASS, 1, 16, 2, L.NIF_F16]
    for word, bad in ((9, L.NIF_ENC_SPHERICAL_OUTER), (10, L.NIF_NETS_OBJECT), (11, 5), (12, 8), (13, 4),
                      (14, L.NIF_F32), (15, 12345)):
        h = np.zeros(64, dtype=np.int64)
        h[:15] = good
        if word < 15:
            h[word] = bad
        else:
            h[15] = bad
        assert L.lib.nif_state_load(ctypes.byref(d), ctypes.byref(o), h.ctypes.data_as(ctypes.c_void_p), size,
                                    None) == L.NIF_ERR_ARG
        assert f"header word {word} " in L.last_error(), (word, L.last_error())


def test_argument_errors_of_the_widened_calls(L):
    """Host-side checks of the primary-ray, lighting, deterministic and
    round-1 additions: every bad argument returns before any work is
    queued (no GPU is needed to see it)."""
    P = ctypes.c_void_p
    assert L.lib.nif_loss_aux(None, None, None, 4, 1, 1.0, None, None, None) == L.NIF_ERR_ARG  # O < 2
    assert L.lib.nif_loss_aux(None, None, None, -1, 5, 1.0, None, None, None) == L.NIF_ERR_ARG
    assert L.lib.nif_loss_aux(None, None, None, 0, 5, 1.0, None, None, None) == L.NIF_OK
    assert L.lib.nif_light_cdf(None, 0, None, None) == L.NIF_ERR_ARG
    assert L.lib.nif_light_samples(None, None, None, None, None, 4, 0, None, None, 1, None, 1e-3, 0.8,
                                   None, None, None) == L.NIF_ERR_ARG          # spp 0
    assert L.lib.nif_light_samples(None, None, None, None, None, 0, 2, None, None, 1, None, 1e-3, 0.8,
                                   None, None, None) == L.NIF_OK               # no rays
    assert L.lib.nif_shade(None, None, -1, 1, None, None) == L.NIF_ERR_ARG
    assert L.lib.nif_bits_clear(None, -1, None) == L.NIF_ERR_ARG
    assert L.lib.nif_bits_clear(None, 0, None) == L.NIF_OK
    assert L.lib.bvh_cast_pairs_closest(None, None, None, None, -1, None, None, None) == L.NIF_ERR_ARG
    assert L.lib.bvh_cast_shadow_or(None, None, -1, None, None) == L.NIF_ERR_ARG
    # five outputs: weights grow by four output rows; too narrow a network refuses them
    d1, d5 = _room_desc(L), _room_desc(L, n_outputs=5)
    assert L.lib.nif_weight_count(ctypes.byref(d5)) - L.lib.nif_weight_count(ctypes.byref(d1)) == 4 * 64
    narrow = _room_desc(L, n_outputs=5, width=4)
    assert L.lib.nif_weight_count(ctypes.byref(narrow)) > 0
    assert L.lib.nif_workspace_size(ctypes.byref(narrow), 10, 10) == 0
    assert L.lib.nif_workspace_size(ctypes.byref(_room_desc(L, n_outputs=9)), 10, 10) == 0
    # the resolution needs the primary-ray layout; a shadow-ray model is refused
    assert L.lib.nif_primary_resolve(ctypes.byref(d1), None, 10, None, None, None, 0, None, None, None, None,
                                     None, None) == L.NIF_ERR_ARG
    assert "5 outputs" in L.last_error()
    # a train step of a five-output network without targets is refused
    o = L.OptimDesc()
    for f in ("d_w_master", "d_w_grad", "d_w_m", "d_w_v", "d_g_master", "d_g_grad", "d_g_m", "d_g_v"):
        setattr(o, f, 256)
    o.loss_scale = 1.0
    assert L.lib.nif_train_step(ctypes.byref(d5), ctypes.byref(o), P(256), P(256), P(256), P(256), P(256), 8,
                                None, P(256), 1 << 20, None) == L.NIF_ERR_ARG
    assert "targets" in L.last_error()
    # round-1 rule: only the two defined values
    assert L.lib.nif_workspace_size(ctypes.byref(_room_desc(L, round1=L.NIF_ROUND1_OUTER)), 10, 10) > 0
    assert L.lib.nif_workspace_size(ctypes.byref(_room_desc(L, round1=7)), 10, 10) == 0
    # deterministic scratch: at least the records (element, value) of every grid tap
    taps = 3 * 16 * 8 * 2
    assert L.lib.nif_deterministic_workspace_size(ctypes.byref(d1), 1000) >= 1000 * taps * 8
    assert L.lib.nif_deterministic_workspace_size(ctypes.byref(d1), -1) == 0


def test_argument_errors_of_the_rate_measurement(L):
    """nif_tc_mma_rate refuses shapes the tensor cores do not take and bad
    counts before touching the device."""
    P = ctypes.c_void_p
    for m, n, a_tmem, chain, reps in ((96, 64, 0, 4, 4), (128, 8, 0, 4, 4), (128, 272, 0, 4, 4),
                                      (64, 256, 1, 4, 4), (128, 64, 0, 0, 4), (128, 64, 0, 4, 0)):
        assert L.lib.nif_tc_mma_rate(m, n, a_tmem, chain, reps, 1, P(256), P(256), 256, None) == L.NIF_ERR_ARG
