"""``python -m paper_2210_03211_gb300 EDGES ...``: see :mod:`paper_2210_03211_gb300.cli`."""
import sys

from .cli import main

sys.exit(main())
