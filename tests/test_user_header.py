"""The user-interaction header template compiles for sm_103a (no GPU)."""
import os

from user_laws_build import compile_object


def test_user_laws_compile_against_the_header():
    obj = compile_object()
    assert os.path.getsize(obj) > 0
