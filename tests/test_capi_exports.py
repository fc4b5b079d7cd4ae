"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function declared in include/aspamg.h (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "aspamg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:\w+\s+)+\**\s*(amg_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("amg_setup", "amg_solve", "amg_adjoint", "amg_update_values", "amg_elem_grad",
                     "amg_get_stats", "amg_free", "amg_strerror", "amg_default_params"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_1902_01715_gb300 as A
    path = A.build()
    L = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert sorted(A.EXPORTS) == declared_functions()


def test_defaults_follow_the_paper_table():
    import paper_1902_01715_gb300 as A
    p = A.default_params()
    # Table TestParam: k_g = 4, eps_g = 1e-3, n_tv = 10, n_rq = 10, theta = 5,
    # n_max = 5, kappa_p = 50 (rho_g counts nodes in the block form)
    assert (p.k_g, p.eps_g, p.n_tv, p.n_rq, p.theta, p.n_max, p.kappa_p) == (4, 1e-3, 10, 10, 5, 5, 50.0)
    assert p.maxit == 1000 and p.vcycle_prec == A.AMG_FP64


def test_oracle_and_library_defaults_agree(orc):
    import paper_1902_01715_gb300 as A
    g, o = A.default_params(), orc.default_params(3)
    for f in ("k_g", "rho_g", "eps_g", "k_i", "rho_i", "eps_i", "omega_bar", "rho_bar", "max_refine",
              "max_g_nodes", "lanczos_m", "omega_safety", "n_tv", "n_rq", "k_ritz", "theta", "n_max",
              "d_p", "kappa_p", "n_coarse", "max_levels", "max_coarse_ratio", "seed"):
        assert getattr(g, f) == getattr(o, f), f
