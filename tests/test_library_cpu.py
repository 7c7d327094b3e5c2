"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every entry point the header declares, validates
configurations, and the state-buffer marshalling round-trips."""

import ctypes
import os
import re

import numpy as np
import pytest

from paper_2505_18519_gb300 import afqmc as lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2505_18519_gb300 import build
    build.build()
    return lib.load_library()


def test_exports_every_declared_symbol(L):
    header = open(os.path.join(ROOT, "include", "afqmc.h")).read()
    declared = set(re.findall(r"\b(afqmc_[a-z_0-9]+)\s*\(", header))
    assert "afqmc_init" in declared and "afqmc_step" in declared and "afqmc_energy" in declared
    for name in declared:
        assert hasattr(L, name), name
    assert declared >= set(lib.EXPORTS)


def test_config_validation(L):
    good = lib.make_config(8, 4, 4, 32, 8, 64, 16, 0.01, 1)
    assert lib.workspace_bytes(good) > 0
    for field, bad in (("N", 0), ("n_up", 0), ("n_dn", 5), ("n_paths", 0), ("dtau", 0.0), ("taylor_order", 0),
                       ("constraint", 7), ("precision", 9), ("n_chol", 0), ("importance", 2), ("importance", -1),
                       ("pop_period", -1)):
        c = lib.make_config(8, 4, 4, 32, 8, 64, 16, 0.01, 1)
        setattr(c, field, bad)
        assert lib.workspace_bytes(c) == 0, field


def test_init_rejects_bad_workspace_without_touching_a_gpu(L):
    c = lib.make_config(8, 4, 4, 32, 8, 4, 2, 0.01, 1)
    out = ctypes.c_void_p()
    h = np.zeros((8, 8))
    st = L.afqmc_init(ctypes.byref(c), h.ctypes.data, h.ctypes.data, h.ctypes.data, h.ctypes.data, None, 0, None,
                      ctypes.byref(out))
    assert st == 3 and out.value is None                     # AFQMC_ERR_WORKSPACE
    st = L.afqmc_init(None, None, None, None, None, None, 0, None, ctypes.byref(out))
    assert st == 1 and b"NULL" in L.afqmc_last_error()      # AFQMC_ERR_ARG


def test_population_control_fields_reach_the_library(L):
    """The two fields appended to the config are read at their offsets: the comb's
    buffers appear in the workspace only with pop_period > 0, and its walker limit
    and the importance functions are checked."""
    base = lib.make_config(8, 4, 4, 32, 8, 64, 16, 0.01, 1)
    le = lib.make_config(8, 4, 4, 32, 8, 64, 16, 0.01, 1, importance="local_energy")
    comb = lib.make_config(8, 4, 4, 32, 8, 64, 16, 0.01, 1, pop_period=5)
    assert lib.workspace_bytes(le) == lib.workspace_bytes(base) > 0
    assert lib.workspace_bytes(comb) > lib.workspace_bytes(base)
    assert lib.workspace_bytes(lib.make_config(8, 4, 4, 32, 8, 65535, 1, 0.01, 1, pop_period=1)) > 0
    assert lib.workspace_bytes(lib.make_config(8, 4, 4, 32, 8, 65536, 1, 0.01, 1, pop_period=1)) == 0
    assert lib.workspace_bytes(lib.make_config(8, 4, 4, 32, 8, 65536, 1, 0.01, 1)) > 0
    d = lib.AfqmcConfig()
    L.afqmc_config_default(ctypes.byref(d))
    assert d.importance == 0 and d.pop_period == 0 and d.refine_tol == 1e-4


def test_half_rotation_cache_configuration(L):
    """rcache = 1 needs FP64 and sizes whose Theta fits four warps' shared memory;
    its workspace holds (n_chol + 1) N n_up doubles per pair more."""
    base = lib.make_config(50, 10, 10, 250, 50, 16, 32, 0.005, 1)
    rc = lib.make_config(50, 10, 10, 250, 50, 16, 32, 0.005, 1, rcache=True)
    extra = lib.workspace_bytes(rc) - lib.workspace_bytes(base)
    assert extra >= 16 * 32 * 251 * 50 * 10 * 8
    assert extra < 16 * 32 * 251 * 50 * 10 * 8 + 16 * 32 * 8 + 4096
    assert lib.workspace_bytes(lib.make_config(50, 10, 10, 250, 50, 16, 32, 0.005, 1, rcache=True,
                                               precision="fp16x3")) == 0
    assert lib.workspace_bytes(lib.make_config(120, 24, 24, 600, 120, 4, 8, 0.005, 1, rcache=True)) == 0
    c = lib.make_config(8, 4, 4, 32, 8, 64, 16, 0.01, 1)
    c.rcache = 2
    assert lib.workspace_bytes(c) == 0
    assert lib.contract_kernel(rc) == "contract_fp64r_kernel"


def test_workspace_grows_with_walkers(L):
    a = lib.workspace_bytes(lib.make_config(50, 10, 10, 250, 50, 16, 32, 0.005, 1))
    b = lib.workspace_bytes(lib.make_config(50, 10, 10, 250, 50, 32, 32, 0.005, 1))
    assert b > a and a % 256 == 0


def test_state_pack_roundtrip():
    rng = np.random.default_rng(0)
    W, P, N, nu, nd, K = 3, 2, 5, 3, 2, 4
    st = dict(step=7, phi_up=rng.normal(size=(W, N, nu)) + 1j * rng.normal(size=(W, N, nu)),
              phi_dn=rng.normal(size=(W, N, nd)) + 1j * rng.normal(size=(W, N, nd)),
              weight=rng.random(W), x=rng.normal(size=(W, P, K)), Phi=rng.normal(size=(W, P, N, nu)))
    back = lib.unpack_state(lib.pack_state(st))
    assert back["step"] == 7
    for k in ("phi_up", "phi_dn", "weight", "x", "Phi"):
        assert np.array_equal(back[k], st[k]), k


def test_tensor_core_form_and_wait_limit_fields_reach_the_library(L):
    """tc_form selects the tensor-core form that afqmc_contract_kernel reports
    (host only), and wait_polls / tc_form are validated at their offsets."""
    kw = dict(precision="fp16x3")
    assert lib.contract_kernel(lib.make_config(50, 10, 10, 250, 50, 8, 32, 0.005, 1, **kw)) == "contract_tcy_kernel"
    assert lib.contract_kernel(lib.make_config(120, 24, 24, 600, 120, 8, 64, 0.005, 1, **kw)) == "contract_tc_kernel"
    assert lib.contract_kernel(lib.make_config(120, 24, 24, 600, 120, 8, 64, 0.005, 1, tc_form="walker",
                                               **kw)) == "contract_tcw_kernel"
    # N = 200 with 40 + 40 electrons: only the general walker-side form takes it
    assert lib.contract_kernel(lib.make_config(200, 40, 40, 1000, 200, 8, 16, 0.005, 1, **kw)) == "contract_tcw_kernel"
    with pytest.raises(lib.AfqmcError):
        lib.contract_kernel(lib.make_config(200, 40, 40, 1000, 200, 8, 16, 0.005, 1, tc_form="per_pair", **kw))
    for field, bad in (("wait_polls", -1), ("wait_polls", (1 << 31) + 1), ("tc_form", 3), ("tc_form", -1)):
        c = lib.make_config(8, 4, 4, 32, 8, 64, 16, 0.01, 1, **kw)
        setattr(c, field, bad)
        assert lib.workspace_bytes(c) == 0, field
    # the general form's work space (its X image and per-chunk images) is in the total
    a = lib.workspace_bytes(lib.make_config(120, 24, 24, 600, 120, 8, 64, 0.005, 1, **kw))
    b = lib.workspace_bytes(lib.make_config(120, 24, 24, 600, 120, 8, 64, 0.005, 1, tc_form="walker", **kw))
    assert a > 0 and b > 0 and a != b


def test_three_part_precision_takes_only_the_general_walker_side_form(L):
    """fp16x6 (three FP16 parts per operand) runs only on the general walker-side
    form, up to N = 256 with n_up <= 40: the auto form picks it, the per-pair form,
    n_up = 48 and N = 264 are refused, and its work space holds three-part images
    (more than fp16x3's)."""
    kw = dict(precision="fp16x6")
    for shape in ((50, 10, 10, 250, 50, 8, 32), (120, 24, 24, 600, 120, 8, 64), (192, 40, 40, 100, 20, 4, 16),
                  (200, 40, 40, 1000, 200, 8, 16), (256, 40, 40, 100, 20, 4, 16)):
        assert lib.contract_kernel(lib.make_config(*shape, 0.005, 1, **kw)) == "contract_tcw_kernel", shape
    with pytest.raises(lib.AfqmcError):
        lib.contract_kernel(lib.make_config(120, 24, 24, 600, 120, 8, 64, 0.005, 1, tc_form="per_pair", **kw))
    for shape in ((128, 48, 48, 100, 20, 4, 16), (264, 40, 40, 100, 20, 4, 16)):
        with pytest.raises(lib.AfqmcError):
            lib.contract_kernel(lib.make_config(*shape, 0.005, 1, **kw))
    a = lib.workspace_bytes(lib.make_config(120, 24, 24, 600, 120, 8, 64, 0.005, 1, tc_form="walker",
                                            precision="fp16x3"))
    b = lib.workspace_bytes(lib.make_config(120, 24, 24, 600, 120, 8, 64, 0.005, 1, **kw))
    assert b > a > 0
    c = lib.make_config(8, 4, 4, 32, 8, 64, 16, 0.01, 1, **kw)
    c.precision = 4
    assert lib.workspace_bytes(c) == 0


def test_trial_fields_reach_the_library(L):
    """The trial's alpha and slice count select the complex-trial contraction, and
    the combinations it does not support are refused (host only)."""
    c = lib.make_config(8, 4, 4, 32, 8, 8, 4, 0.01, 1, trial_alpha=-0.5j, trial_slices=2)
    assert lib.contract_kernel(c) == "contract_fp64c_kernel"
    real = lib.make_config(8, 4, 4, 32, 8, 8, 4, 0.01, 1)
    assert lib.workspace_bytes(c) > lib.workspace_bytes(real)        # complex Phi, slice buffers
    for kw in (dict(precision="fp16x3", tc_form="per_pair"), dict(proposal="mlp"), dict(rcache=True),
               dict(trial_slices=9), dict(trial_alpha=0.0)):
        bad = lib.make_config(8, 4, 4, 32, 8, 8, 4, 0.01, 1, **{"trial_alpha": -0.5j, **kw})
        assert lib.workspace_bytes(bad) == 0, kw
    # mixed precision: the walker-side tensor-core form, whatever the requested form
    for prec in ("fp16x3", "fp16x6", "bf16x3"):
        m = lib.make_config(8, 4, 4, 32, 8, 8, 4, 0.01, 1, trial_alpha=-0.5j, trial_slices=2, precision=prec)
        assert lib.contract_kernel(m) == "contract_tcw_kernel"
        assert lib.workspace_bytes(m) > 0


def test_trial_form_field_reaches_the_library(L):
    """trial_form selects how the mixed path forms exp(S) Phi0; an unknown value is refused."""
    for form in ("auto", "df", "tc"):
        c = lib.make_config(50, 10, 10, 250, 50, 4, 8, 0.005, 1, precision="fp16x6", trial_form=form)
        assert lib.workspace_bytes(c) > 0
    c = lib.make_config(50, 10, 10, 250, 50, 4, 8, 0.005, 1, precision="fp16x6")
    c.trial_form = 7
    assert lib.workspace_bytes(c) == 0


def test_overlap_form_field_reaches_the_library(L):
    """overlap_form selects how the mixed path forms the overlap matrices: the
    tensor-core form holds them in the work space (16 bytes per entry, both spins),
    the double-float form does not; an unknown value is refused."""
    N, nu, nd, W, P = 120, 24, 24, 8, 16
    a = lib.workspace_bytes(lib.make_config(N, nu, nd, 600, N, W, P, 0.005, 1, precision="fp16x6"))
    d = lib.workspace_bytes(lib.make_config(N, nu, nd, 600, N, W, P, 0.005, 1, precision="fp16x6",
                                            overlap_form="df"))
    assert a - d >= W * P * (nu * nu + nd * nd) * 16
    assert a - d < W * P * (nu * nu + nd * nd) * 16 + 512
    # beyond the tensor-core form's sizes (N > 128) both forms are the double-float one
    big = [lib.workspace_bytes(lib.make_config(200, 40, 40, 1000, 200, 4, 4, 0.005, 1, precision="fp16x6",
                                               overlap_form=f)) for f in ("auto", "df")]
    assert big[0] == big[1] > 0
    c = lib.make_config(N, nu, nd, 600, N, W, P, 0.005, 1, precision="fp16x6")
    c.overlap_form = 3
    assert lib.workspace_bytes(c) == 0
