"""python -m paper_2510_25938_gb300 input.molden -- see cli.py."""
import sys

from .cli import main

sys.exit(main())
